/*
 * CPU FP64 oracle for the density-matrix problem.  TEST INFRASTRUCTURE ONLY: the product path
 * never links, loads or calls this file; only the tests, the smoke check and the bench's CPU
 * baseline do.
 *
 * What it computes is the plain definition of the result, not the GPU method:
 *   - the generalised eigenproblem H C = S C eps               (Sec. 1, Eq. evp)
 *   - orthogonalisation by the Loewdin factor S^{-1/2}:
 *       H~ = S^{-1/2} H S^{-1/2}                              (Sec. 2.2.2, Eq. ntpoly_lowdin)
 *   - the zero-temperature density matrix p_ij = sum_l f_l c_il c_jl with f_l = 1 for the
 *     n_occ lowest eps and 0 otherwise                         (Sec. 1, Eq. density_matrix)
 * Eigenpairs come from a two-sided cyclic Jacobi method (plain rotations, no blocking), applied
 * once to S and once to H~:  S = U diag(s) U^T,  Z = U diag(s^{-1/2}) U^T,  H~ = Z H Z,
 * H~ = V diag(lam) V^T,  C_occ = Z V[:, :n_occ],  P = C_occ C_occ^T,  E = sum_{l<n_occ} lam_l.
 *
 * The rotations inside one round act on disjoint index pairs (round-robin ordering), which is
 * the same Jacobi method in a different pair order; it lets OpenMP run the pairs of a round in
 * parallel.  Nothing here is shared with the CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_NOT_SPD = 3, OR_NO_GAP = 5, OR_NOT_CONVERGED = 6, OR_OOM = 7 };

/* ---------------------------------------------------------------------------------------- */
/* plain dense helpers, row-major n x n unless stated                                        */
/* ---------------------------------------------------------------------------------------- */

/* C (m x p) = A (m x k) * B (k x p), all row-major with the given leading dimensions. */
static void mat_mul(int64_t m, int64_t k, int64_t p, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double *C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double *c = C + i * ldc;
        for (int64_t j = 0; j < p; ++j) c[j] = 0.0;
        for (int64_t l = 0; l < k; ++l) {
            const double a = A[i * lda + l];
            const double *b = B + l * ldb;
            for (int64_t j = 0; j < p; ++j) c[j] += a * b[j];
        }
    }
}

static void symmetrise(int64_t n, double *A) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            const double v = 0.5 * (A[i * n + j] + A[j * n + i]);
            A[i * n + j] = v;
            A[j * n + i] = v;
        }
}

/* ---------------------------------------------------------------------------------------- */
/* two-sided cyclic Jacobi                                                                   */
/* ---------------------------------------------------------------------------------------- */

/* Pairs of round r of a round-robin tournament on m (even) players; player m-1 stays put and
 * the others rotate.  Writes m/2 pairs (p < q) into pp/qq. */
static void round_robin_pairs(int64_t m, int64_t r, int64_t *pp, int64_t *qq) {
    const int64_t half = m / 2;
    for (int64_t k = 0; k < half; ++k) {
        int64_t a, b;
        if (k == 0) {
            a = m - 1;
            b = r % (m - 1);
        } else {
            a = (r + k) % (m - 1);
            b = (r + (m - 1) - k) % (m - 1);
        }
        pp[k] = a < b ? a : b;
        qq[k] = a < b ? b : a;
    }
}

/*
 * Eigen-decomposition of the symmetric n x n matrix A (row-major; destroyed).
 * On return evals[0..n) ascending (ties kept in index order) and column l of V (row-major,
 * V[i*n + l]) is the unit eigenvector of evals[l].  Stops when the off-diagonal Frobenius norm
 * is <= tol * ||A||_F or after max_sweeps sweeps.  Returns OR_OK or OR_NOT_CONVERGED.
 */
int oracle_jacobi_eigh(int64_t n, double *A, double *evals, double *V, double tol,
                       int max_sweeps, int *sweeps_out) {
    if (n <= 0 || !A || !evals || !V) return OR_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    symmetrise(n, A);

    double fro2 = 0.0;
    for (int64_t i = 0; i < n * n; ++i) fro2 += A[i] * A[i];
    const double target = tol * tol * fro2;

    const int64_t m = (n % 2 == 0) ? n : n + 1; /* a dummy player when n is odd */
    const int64_t half = m / 2;
    int64_t *pp = (int64_t *)malloc(sizeof(int64_t) * half);
    int64_t *qq = (int64_t *)malloc(sizeof(int64_t) * half);
    double *cs = (double *)malloc(sizeof(double) * half);
    double *sn = (double *)malloc(sizeof(double) * half);
    if (!pp || !qq || !cs || !sn) {
        free(pp); free(qq); free(cs); free(sn);
        return OR_OOM;
    }

    int status = OR_NOT_CONVERGED;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off2 = 0.0;
#pragma omp parallel for reduction(+ : off2) schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j)
                if (i != j) off2 += A[i * n + j] * A[i * n + j];
        if (off2 <= target) {
            status = OR_OK;
            break;
        }
        for (int64_t r = 0; r < m - 1; ++r) {
            round_robin_pairs(m, r, pp, qq);
            /* angles from the current A: each pair's 2x2 block is touched only by its own
             * rotation within the round, because the pairs are disjoint */
            for (int64_t k = 0; k < half; ++k) {
                const int64_t p = pp[k], q = qq[k];
                cs[k] = 1.0;
                sn[k] = 0.0;
                if (q >= n) continue; /* dummy */
                const double apq = A[p * n + q];
                if (apq == 0.0) continue;
                const double app = A[p * n + p], aqq = A[q * n + q];
                /* symmetric Schur 2x2: t = tan(theta) zeroes the (p,q) entry of J^T A J */
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                               : -1.0 / (-tau + sqrt(1.0 + tau * tau));
                cs[k] = 1.0 / sqrt(1.0 + t * t);
                sn[k] = t * cs[k];
            }
            /* rows: A <- J^T A   (rows p, q of each pair) */
#pragma omp parallel for schedule(static)
            for (int64_t k = 0; k < half; ++k) {
                const int64_t p = pp[k], q = qq[k];
                if (q >= n || sn[k] == 0.0) continue;
                const double c = cs[k], s = sn[k];
                double *ap = A + p * n, *aq = A + q * n;
                for (int64_t j = 0; j < n; ++j) {
                    const double x = ap[j], y = aq[j];
                    ap[j] = c * x - s * y;
                    aq[j] = s * x + c * y;
                }
            }
            /* columns: A <- A J and V <- V J   (columns p, q of each pair, row by row) */
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                double *ai = A + i * n, *vi = V + i * n;
                for (int64_t k = 0; k < half; ++k) {
                    const int64_t p = pp[k], q = qq[k];
                    if (q >= n || sn[k] == 0.0) continue;
                    const double c = cs[k], s = sn[k];
                    double x = ai[p], y = ai[q];
                    ai[p] = c * x - s * y;
                    ai[q] = s * x + c * y;
                    x = vi[p];
                    y = vi[q];
                    vi[p] = c * x - s * y;
                    vi[q] = s * x + c * y;
                }
            }
            for (int64_t k = 0; k < half; ++k) {
                const int64_t p = pp[k], q = qq[k];
                if (q >= n || sn[k] == 0.0) continue;
                A[p * n + q] = 0.0;
                A[q * n + p] = 0.0;
            }
        }
    }
    if (sweeps_out) *sweeps_out = sweep;

    /* ascending order, ties by index (insertion sort on a permutation: n is small here) */
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * n);
    double *tmp = (double *)malloc(sizeof(double) * n * n);
    if (!perm || !tmp) {
        free(perm); free(tmp); free(pp); free(qq); free(cs); free(sn);
        return OR_OOM;
    }
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t i = 1; i < n; ++i) {
        const int64_t key = perm[i];
        const double kv = A[key * n + key];
        int64_t j = i - 1;
        while (j >= 0 && A[perm[j] * n + perm[j]] > kv) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = key;
    }
    for (int64_t l = 0; l < n; ++l) evals[l] = A[perm[l] * n + perm[l]];
    memcpy(tmp, V, sizeof(double) * n * n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t l = 0; l < n; ++l) V[i * n + l] = tmp[i * n + perm[l]];
    free(perm); free(tmp); free(pp); free(qq); free(cs); free(sn);
    return status;
}

/* ---------------------------------------------------------------------------------------- */
/* Loewdin factor and density matrix                                                         */
/* ---------------------------------------------------------------------------------------- */

/* Z = S^{-1/2} through S = U diag(s) U^T (Sec. 2.2.2, Eq. ntpoly_lowdin).  S is symmetrised
 * first.  Returns OR_NOT_SPD if min s <= 0; s_min/s_max are reported when non-NULL. */
int oracle_inv_sqrt(int64_t n, const double *S, double *Z, double *s_min, double *s_max) {
    if (n <= 0 || !S || !Z) return OR_ERR_ARG;
    double *A = (double *)malloc(sizeof(double) * n * n);
    double *U = (double *)malloc(sizeof(double) * n * n);
    double *w = (double *)malloc(sizeof(double) * n);
    double *US = (double *)malloc(sizeof(double) * n * n);
    double *UT = (double *)malloc(sizeof(double) * n * n);
    if (!A || !U || !w || !US || !UT) {
        free(A); free(U); free(w); free(US); free(UT);
        return OR_OOM;
    }
    memcpy(A, S, sizeof(double) * n * n);
    int sweeps = 0;
    int st = oracle_jacobi_eigh(n, A, w, U, 1e-15, 60, &sweeps);
    if (s_min) *s_min = w[0];
    if (s_max) *s_max = w[n - 1];
    if (st == OR_OK && w[0] <= 0.0) st = OR_NOT_SPD;
    if (st == OR_OK) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t l = 0; l < n; ++l) {
                US[i * n + l] = U[i * n + l] / sqrt(w[l]);
                UT[l * n + i] = U[i * n + l];
            }
        mat_mul(n, n, n, US, n, UT, n, Z, n);
        symmetrise(n, Z);
    }
    free(A); free(U); free(w); free(US); free(UT);
    return st;
}

/*
 * Energy-weighted density matrix q_ij = sum_l f_l eps_l c_il c_jl (Sec. 2.6, Eq.
 * energy_density_matrix) from C_occ (n x n_occ, leading dimension n_occ) and eps.
 */
static void energy_weighted(int64_t n, int64_t n_occ, const double *C, const double *eps,
                            double *Q) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t l = 0; l < n_occ; ++l) acc += eps[l] * C[i * n_occ + l] * C[j * n_occ + l];
            Q[i * n + j] = acc;
        }
    symmetrise(n, Q);
}

/*
 * Zero-temperature density matrix of (H, S) with n_occ occupied states (f_l in {0, 1}).
 * Outputs: P (n x n), *energy = sum of the n_occ lowest generalised eigenvalues = Tr(P H),
 * *trace_ps = Tr(P S), *idem = ||P S P - P||_F, *gap = lam[n_occ] - lam[n_occ-1] (0 if n_occ
 * is 0 or n), evals (optional, n ascending generalised eigenvalues).
 * Returns OR_OK, OR_NOT_SPD, OR_NO_GAP (outputs still written) or OR_NOT_CONVERGED.
 */
int oracle_density_matrix_edm(int64_t n, int64_t n_occ, const double *H_in,
                              const double *S_in, double *P, double *energy, double *trace_ps,
                              double *idem, double *gap, double *evals, double *Q);

int oracle_density_matrix(int64_t n, int64_t n_occ, const double *H_in, const double *S_in,
                          double *P, double *energy, double *trace_ps, double *idem,
                          double *gap, double *evals) {
    return oracle_density_matrix_edm(n, n_occ, H_in, S_in, P, energy, trace_ps, idem, gap, evals,
                                     NULL);
}

/* As oracle_density_matrix, plus the energy-weighted density matrix Q (n x n) when Q != NULL. */
int oracle_density_matrix_edm(int64_t n, int64_t n_occ, const double *H_in,
                              const double *S_in, double *P, double *energy, double *trace_ps,
                              double *idem, double *gap, double *evals, double *Q) {
    if (n <= 0 || n_occ < 0 || n_occ > n || !H_in || !S_in || !P) return OR_ERR_ARG;
    const size_t nn = (size_t)n * (size_t)n;
    double *H = (double *)malloc(sizeof(double) * nn);
    double *S = (double *)malloc(sizeof(double) * nn);
    double *Z = (double *)malloc(sizeof(double) * nn);
    double *T = (double *)malloc(sizeof(double) * nn);
    double *Ht = (double *)malloc(sizeof(double) * nn);
    double *V = (double *)malloc(sizeof(double) * nn);
    double *lam = (double *)malloc(sizeof(double) * n);
    if (!H || !S || !Z || !T || !Ht || !V || !lam) {
        free(H); free(S); free(Z); free(T); free(Ht); free(V); free(lam);
        return OR_OOM;
    }
    memcpy(H, H_in, sizeof(double) * nn);
    memcpy(S, S_in, sizeof(double) * nn);
    symmetrise(n, H); /* reading: inputs are symmetrised on ingest */
    symmetrise(n, S);

    int st = oracle_inv_sqrt(n, S, Z, NULL, NULL);
    if (st != OR_OK) goto done;

    /* H~ = Z H Z (Eq. ntpoly_lowdin) */
    mat_mul(n, n, n, Z, n, H, n, T, n);
    mat_mul(n, n, n, T, n, Z, n, Ht, n);
    symmetrise(n, Ht);

    int sweeps = 0;
    st = oracle_jacobi_eigh(n, Ht, lam, V, 1e-15, 60, &sweeps);
    if (st != OR_OK) goto done;
    if (evals) memcpy(evals, lam, sizeof(double) * n);

    /* C_occ = Z V[:, :n_occ]  (n x n_occ, stored in T with leading dimension n) */
    if (n_occ > 0) {
        /* Vo = V[:, :n_occ] gathered into Ht (free now) */
        for (int64_t i = 0; i < n; ++i)
            for (int64_t l = 0; l < n_occ; ++l) Ht[i * n_occ + l] = V[i * n + l];
        mat_mul(n, n, n_occ, Z, n, Ht, n_occ, T, n_occ);
        /* P = C_occ C_occ^T */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double acc = 0.0;
                for (int64_t l = 0; l < n_occ; ++l) acc += T[i * n_occ + l] * T[j * n_occ + l];
                P[i * n + j] = acc;
            }
        symmetrise(n, P);
        if (Q) energy_weighted(n, n_occ, T, lam, Q);
    } else {
        memset(P, 0, sizeof(double) * nn);
        if (Q) memset(Q, 0, sizeof(double) * nn);
    }

    double e = 0.0;
    for (int64_t l = 0; l < n_occ; ++l) e += lam[l];
    if (energy) *energy = e;
    if (gap) *gap = (n_occ > 0 && n_occ < n) ? lam[n_occ] - lam[n_occ - 1] : 0.0;

    if (trace_ps) {
        double t = 0.0;
        for (size_t i = 0; i < nn; ++i) t += P[i] * S[i];
        *trace_ps = t;
    }
    if (idem) {
        /* ||P S P - P||_F */
        mat_mul(n, n, n, P, n, S, n, T, n);
        mat_mul(n, n, n, T, n, P, n, V, n);
        double d = 0.0;
        for (size_t i = 0; i < nn; ++i) d += (V[i] - P[i]) * (V[i] - P[i]);
        *idem = sqrt(d);
    }
    /* a gap below 1e-12 of the spectral width is rounding noise: the occupied subspace is not
     * unique and several P would be correct */
    if (n_occ > 0 && n_occ < n &&
        lam[n_occ] - lam[n_occ - 1] <= 1e-12 * (fabs(lam[n - 1] - lam[0]) + 1e-300))
        st = OR_NO_GAP;

done:
    free(H); free(S); free(Z); free(T); free(Ht); free(V); free(lam);
    return st;
}

/* number of OpenMP threads this library uses (1 without OpenMP) */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
