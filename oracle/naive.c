/* The definition of Eq. ShiftInvariance as literal loops, plain C, float64.
 * TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
 *
 * F:  [N_t][N_d][N_m] first block column, F[k] = F_{k} (0-based lag).
 * m:  [N_t][N_m], d: [N_t][N_d] (time-outer).
 *
 * oracle_naive_forward:  d_i[s] = sum_{j<=i} sum_l F_{i-j}[s][l] m_j[l]
 * oracle_naive_adjoint:  m_j[l] = sum_{i>=j} sum_s F_{i-j}[s][l] d_i[s]
 */
#include <stddef.h>

void oracle_naive_forward(int N_t, int N_d, int N_m, const double* F, const double* m, double* d)
{
    for (int i = 0; i < N_t; ++i)
        for (int s = 0; s < N_d; ++s) {
            double acc = 0.0;
            for (int j = 0; j <= i; ++j) {
                const double* Fk = F + (size_t)(i - j) * N_d * N_m + (size_t)s * N_m;
                const double* mj = m + (size_t)j * N_m;
                for (int l = 0; l < N_m; ++l) acc += Fk[l] * mj[l];
            }
            d[(size_t)i * N_d + s] = acc;
        }
}

void oracle_naive_adjoint(int N_t, int N_d, int N_m, const double* F, const double* d, double* m)
{
    for (int j = 0; j < N_t; ++j)
        for (int l = 0; l < N_m; ++l) {
            double acc = 0.0;
            for (int i = j; i < N_t; ++i)
                for (int s = 0; s < N_d; ++s)
                    acc += F[(size_t)(i - j) * N_d * N_m + (size_t)s * N_m + l] * d[(size_t)i * N_d + s];
            m[(size_t)j * N_m + l] = acc;
        }
}
