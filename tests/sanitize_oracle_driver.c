/* Exercises every entry point of oracle/dtw_oracle.c on seeded inputs of many
 * sizes (n = 1 .. 70, w from 0 to beyond n, k beyond N, every p and cascade
 * mode) so that a build under AddressSanitizer and UndefinedBehaviorSanitizer
 * reports any out-of-bounds access, leak or undefined operation.  Exit 0 when
 * every call ran; results are checked elsewhere (test_oracle_pins.py). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void oracle_envelope_d(const double *y, int64_t n, int64_t w, double *U, double *L);
void oracle_envelope(const float *y, int64_t n, int64_t w, double *U, double *L);
void oracle_projection(const double *x, const double *U, const double *L, int64_t n, double *H);
double oracle_lb_keogh_pow_d(const double *x, const double *U, const double *L, int64_t n, int p);
double oracle_lb_keogh_pow(const float *x, const double *U, const double *L, int64_t n, int p);
double oracle_lb_improved_pow(const float *x, const float *y, const double *U, const double *L, int64_t n,
                              int64_t w, int p, double *first_pass);
double oracle_dtw_pow(const float *x, const float *y, int64_t n, int64_t w, int p);
double oracle_lb_piecewise_pow(const float *x, const double *U, const double *L, int64_t n, int64_t d, int p);
void oracle_knn_bruteforce(const float *db, int64_t N, const float *y, int64_t n, int64_t w, int p, int k,
                           int64_t *out_idx, double *out_dist);
void oracle_knn_cascade(const float *db, int64_t N, const float *y, int64_t n, int64_t w, int p, int k, int mode,
                        int64_t *out_idx, double *out_dist, int64_t *stats);

static uint64_t state = 0x9E3779B97F4A7C15ull;
static float next_value(void) {  /* xorshift64*, uniform in [-4, 4) */
    state ^= state >> 12;
    state ^= state << 25;
    state ^= state >> 27;
    const uint64_t r = state * 0x2545F4914F6CDD1Dull;
    return (float)((double)(r >> 11) / 9007199254740992.0 * 8.0 - 4.0);
}

int main(void) {
    double sink = 0.0;
    for (int64_t n = 1; n <= 70; n += (n < 10 ? 1 : 7)) {
        const int64_t N = 9;
        float *db = malloc((size_t)(N * n) * sizeof(float));
        float *y = malloc((size_t)n * sizeof(float));
        double *yd = malloc((size_t)n * sizeof(double));
        double *U = malloc((size_t)n * sizeof(double));
        double *L = malloc((size_t)n * sizeof(double));
        double *H = malloc((size_t)n * sizeof(double));
        for (int64_t i = 0; i < N * n; ++i) db[i] = next_value();
        for (int64_t i = 0; i < n; ++i) {
            y[i] = next_value();
            yd[i] = y[i];
        }
        const int64_t bands[] = {0, 1, n / 10, n / 2, n - 1, n, n + 3};
        for (int b = 0; b < 7; ++b) {
            const int64_t w = bands[b];
            oracle_envelope(y, n, w, U, L);
            oracle_envelope_d(yd, n, w, U, L);
            for (int p = 0; p <= 2; ++p) sink += oracle_dtw_pow(db, y, n, w, p);
            for (int p = 1; p <= 2; ++p) {
                double first = 0.0;
                oracle_projection(yd, U, L, n, H);
                sink += oracle_lb_keogh_pow_d(H, U, L, n, p);
                sink += oracle_lb_keogh_pow(db, U, L, n, p);
                sink += oracle_lb_improved_pow(db, y, U, L, n, w, p, &first) + first;
                for (int64_t d = 1; d <= n; d += (d < 4 ? 1 : n / 3 + 1)) sink += oracle_lb_piecewise_pow(db, U, L, n, d, p);
                for (int k = 1; k <= 12; k += 5) {
                    int64_t idx[12], stats[4];
                    double dist[12];
                    oracle_knn_bruteforce(db, N, y, n, w, p, k, idx, dist);
                    for (int mode = 0; mode <= 1; ++mode) oracle_knn_cascade(db, N, y, n, w, p, k, mode, idx, dist, stats);
                    sink += dist[0];
                }
            }
        }
        free(db);
        free(y);
        free(yd);
        free(U);
        free(L);
        free(H);
    }
    printf("ok %g\n", sink);
    return 0;
}
