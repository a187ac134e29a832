/*
 * FP64 reference loop for the static polarizability on the real-space grid.
 *
 * TEST INFRASTRUCTURE ONLY: this file is the oracle's plain C loop.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the GPU library never
 * links or calls it.
 *
 * It evaluates Eq. (Pstatic) of Kim et al., "Scalable GW software for quasiparticle properties
 * using OpenAtom" (Sec. 2, the static omega = 0 polarizability), element by element, with the
 * orientation
 *
 *     P(r, r') = sum_v sum_c 2 conj(psi_v(r)) psi_c(r) conj(psi_c(r')) psi_v(r') / (E_v - E_c)
 *
 * (spin sums folded into the factor 2, q = 0, one k-point).  Energies are in Hartree.
 * psi is complex128, state-major: psi[n * nr + r], occupied states first.
 */
#include <complex.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Rows [r0, r1) of P, written to out[(r - r0) * nr + r'].  Returns 0, or -1 on bad sizes. */
int oracle_P_rows(int nr, int nv, int nc, const double complex *psi, const double *E_ha,
                  int r0, int r1, double complex *out)
{
    if (nr <= 0 || nv <= 0 || nc <= 0 || r0 < 0 || r1 > nr || r0 > r1)
        return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = r0; r < r1; ++r) {
        for (int rp = 0; rp < nr; ++rp) {
            double complex acc = 0.0;
            for (int v = 0; v < nv; ++v) {
                const double complex *pv = psi + (size_t)v * nr;
                for (int c = 0; c < nc; ++c) {
                    const double complex *pc = psi + (size_t)(nv + c) * nr;
                    acc += 2.0 * conj(pv[r]) * pc[r] * conj(pc[rp]) * pv[rp]
                           / (E_ha[v] - E_ha[nv + c]);
                }
            }
            out[(size_t)(r - r0) * nr + rp] = acc;
        }
    }
    return 0;
}
