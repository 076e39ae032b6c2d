/*
 * msd_oracle.c -- plain FP64 CPU oracle for the multi-Slater-determinant wavefunction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or helper with the CUDA library: it has its own
 * problem struct, basis evaluator, LU and sums.
 *
 * It computes the plain definitions, never the table method:
 *   Psi(R)             = sum_I c_I det M_up,I(R) det M_dn,I(R)        (Section II, eq. for Psi)
 *   M_s,I(r, c)        = phi_{col_I(c)}(r_r)                          (Section II, M(i,j) = phi_j(r_i))
 *   Psi(R')/Psi(R)     by two full evaluations                        (Section II, ratio of one move)
 *   grad_i Psi / Psi   and  lap_i Psi / Psi: a determinant is linear in row i, so
 *                      d^a det M = det(M with row i -> d^a phi(r_i))  (Section IV-A, det M^alpha)
 * Every determinant is formed explicitly and factorised by LU with partial pivoting.
 * Each distinct per-spin determinant is computed once per configuration and each term
 * I multiplies one up and one down determinant.
 *
 * Column convention of an excitation string (the paper fixes only M(i,j) = phi_j(r_i)):
 * holes h_1 < ... < h_k of the occupied orbitals 0..n-1 are replaced IN PLACE by the
 * virtual orbitals n + p_1 < ... < n + p_k, i.e. column h_q holds orbital n + p_q.
 *
 * Basis: unnormalised Cartesian Gaussians x^l exp(-alpha |r - A|^2), l <= 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_in_parallel(void) { return 1; }
#endif

typedef struct {
    int32_t n_elec[2], n_orb[2];
    int32_t n_nuc;
    const double* nuc_xyz;      /* [n_nuc][3] */
    int32_t n_basis;
    const int32_t* bas_center;  /* [n_basis] */
    const int8_t* bas_lm;       /* 0 = s, 1 = px, 2 = py, 3 = pz */
    const double* bas_alpha;    /* [n_basis] */
    const double* B[2];         /* per spin [n_basis][n_orb] */
    int32_t n_exc[2];
    const int32_t* exc_off[2];  /* [n_exc + 1] */
    const uint8_t* exc_holes[2];
    const uint8_t* exc_parts[2];
    int64_t n_det;
    const int32_t* det_up;
    const int32_t* det_dn;
    const double* ci;
} orc_problem;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Determinant of the n x n row-major matrix a (destroyed) by LU with partial pivoting.
 * Returns log|det| and sign; a singular matrix gives sign 0 and log|det| = -inf. */
void orc_lu_logdet(int n, double* a, double* logabs, double* sign) {
    double la = 0.0, sg = 1.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = fabs(a[(size_t)r * n + k]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) { *logabs = -INFINITY; *sign = 0.0; return; }
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
            sg = -sg;
        }
        double piv = a[(size_t)k * n + k];
        la += log(fabs(piv));
        if (piv < 0.0) sg = -sg;
        for (int r = k + 1; r < n; ++r) {
            double f = a[(size_t)r * n + k] / piv;
            for (int j = k + 1; j < n; ++j) a[(size_t)r * n + j] -= f * a[(size_t)k * n + j];
        }
    }
    *logabs = la;
    *sign = sg;
}

/* Inverse of the n x n row-major matrix a by LU with partial pivoting and n solves.
 * inv receives A^{-1} (row-major).  Returns 1 if singular. */
static int lu_inverse(int n, const double* a_in, double* lu, int* perm, double* inv, double* col) {
    memcpy(lu, a_in, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(lu[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = fabs(lu[(size_t)r * n + k]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) return 1;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = lu[(size_t)k * n + j];
                lu[(size_t)k * n + j] = lu[(size_t)p * n + j];
                lu[(size_t)p * n + j] = t;
            }
            int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double f = lu[(size_t)r * n + k] / lu[(size_t)k * n + k];
            lu[(size_t)r * n + k] = f;
            for (int j = k + 1; j < n; ++j) lu[(size_t)r * n + j] -= f * lu[(size_t)k * n + j];
        }
    }
    /* solve A x = e_c for each column c: P A = L U */
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) col[i] = (perm[i] == c) ? 1.0 : 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) col[i] -= lu[(size_t)i * n + j] * col[j];
        for (int i = n - 1; i >= 0; --i) {
            for (int j = i + 1; j < n; ++j) col[i] -= lu[(size_t)i * n + j] * col[j];
            col[i] /= lu[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = col[i];
    }
    return 0;
}

/* Basis functions and their derivatives at r: chi[a * n_basis + mu],
 * a = 0 value, 1..3 d/dx, d/dy, d/dz, 4 laplacian. */
void orc_basis(const orc_problem* p, const double* r, double* chi) {
    const int nb = p->n_basis;
    for (int mu = 0; mu < nb; ++mu) {
        const double* A = p->nuc_xyz + 3 * p->bas_center[mu];
        const double al = p->bas_alpha[mu];
        const double d[3] = {r[0] - A[0], r[1] - A[1], r[2] - A[2]};
        const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double g = exp(-al * d2);
        const int lm = p->bas_lm[mu];
        if (lm == 0) {
            /* g; grad g = -2 al d g; lap g = (4 al^2 d2 - 6 al) g */
            chi[0 * nb + mu] = g;
            for (int a = 0; a < 3; ++a) chi[(1 + a) * nb + mu] = -2.0 * al * d[a] * g;
            chi[4 * nb + mu] = (4.0 * al * al * d2 - 6.0 * al) * g;
        } else {
            /* x_c g; d_a (x_c g) = (delta_ac - 2 al d_a d_c) g; lap = d_c (4 al^2 d2 - 10 al) g */
            const int c = lm - 1;
            chi[0 * nb + mu] = d[c] * g;
            for (int a = 0; a < 3; ++a)
                chi[(1 + a) * nb + mu] = ((a == c ? 1.0 : 0.0) - 2.0 * al * d[a] * d[c]) * g;
            chi[4 * nb + mu] = d[c] * (4.0 * al * al * d2 - 10.0 * al) * g;
        }
    }
}

/* Orbitals of spin s at r: phi[a * N + j] = sum_mu chi[a][mu] B_s[mu][j], 5 channels. */
void orc_orbitals(const orc_problem* p, int s, const double* r, double* phi) {
    const int nb = p->n_basis, N = p->n_orb[s];
    double* chi = (double*)malloc(sizeof(double) * 5 * nb);
    orc_basis(p, r, chi);
    for (int a = 0; a < 5; ++a)
        for (int j = 0; j < N; ++j) {
            double acc = 0.0;
            for (int mu = 0; mu < nb; ++mu) acc += chi[a * nb + mu] * p->B[s][(size_t)mu * N + j];
            phi[a * N + j] = acc;
        }
    free(chi);
}

/* Reference Slater matrix of spin s at R: A0[r * n + c] = phi_c(r_r), c < n (Section II). */
void orc_slater(const orc_problem* p, int s, const double* R, double* A0) {
    const int n = p->n_elec[s], N = p->n_orb[s];
    const int off = s ? p->n_elec[0] : 0;
    double* tmp = (double*)malloc(sizeof(double) * 5 * (size_t)N);
    for (int r = 0; r < n; ++r) {
        orc_orbitals(p, s, R + 3 * (off + r), tmp);
        memcpy(A0 + (size_t)r * n, tmp, sizeof(double) * n);
    }
    free(tmp);
}

/* Orbital index held by column c of the determinant of string u (in-place replacement). */
static void string_columns(const orc_problem* p, int s, int u, int* cols) {
    const int n = p->n_elec[s];
    for (int c = 0; c < n; ++c) cols[c] = c;
    const int b = p->exc_off[s][u], e = p->exc_off[s][u + 1];
    for (int q = b; q < e; ++q) cols[p->exc_holes[s][q]] = n + p->exc_parts[s][q];
}

/* Log-determinants of every string of spin s at the n electron positions.
 * phi_rows[r * N + j] = phi_j(r_r).  If drow != NULL, additionally the four matrices with
 * row `row` replaced by drow[a * N + .] (a = 0..3: d/dx, d/dy, d/dz, laplacian). */
static void spin_logdets(const orc_problem* p, int s, const double* phi_rows, int row,
                         const double* drow, double* l, double* sg, double* ld, double* sgd) {
    const int n = p->n_elec[s], N = p->n_orb[s], ne = p->n_exc[s];
#pragma omp parallel if (!omp_in_parallel())
    {
        double* A = (double*)malloc(sizeof(double) * (size_t)n * n);
        int* cols = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
        for (int u = 0; u < ne; ++u) {
            string_columns(p, s, u, cols);
            for (int r = 0; r < n; ++r)
                for (int c = 0; c < n; ++c) A[(size_t)r * n + c] = phi_rows[(size_t)r * N + cols[c]];
            orc_lu_logdet(n, A, &l[u], &sg[u]);
            if (drow) {
                for (int a = 0; a < 4; ++a) {
                    for (int r = 0; r < n; ++r)
                        for (int c = 0; c < n; ++c)
                            A[(size_t)r * n + c] = (r == row) ? drow[a * N + cols[c]]
                                                              : phi_rows[(size_t)r * N + cols[c]];
                    orc_lu_logdet(n, A, &ld[(size_t)a * ne + u], &sgd[(size_t)a * ne + u]);
                }
            }
        }
        free(A);
        free(cols);
    }
}

/*
 * Psi at configuration R ([n_tot][3], up electrons first).  Outputs log|Psi| and sign.
 * If elec >= 0: grad[3] = grad_elec Psi / Psi and lap[0] = lap_elec Psi / Psi.
 * absum (5 doubles, optional): sum_I |c_I X_I| / |Psi| for X = Psi's term (a = 0) and
 * for the four derivative terms (a = 1..4) -- the cancellation scale of each result.
 * Returns 0, or 1 if Psi is exactly zero.
 */
int orc_eval(const orc_problem* p, const double* R, int elec, double* logabs, double* sign,
             double* grad, double* lap, double* absum) {
    double* l[2];
    double* sg[2];
    double* ld = NULL;
    double* sgd = NULL;
    int se = -1, ie = -1;
    if (elec >= 0) {
        se = elec < p->n_elec[0] ? 0 : 1;
        ie = se ? elec - p->n_elec[0] : elec;
    }
    for (int s = 0; s < 2; ++s) {
        const int n = p->n_elec[s], N = p->n_orb[s], ne = p->n_exc[s];
        const int off = s ? p->n_elec[0] : 0;
        double* rows = (double*)malloc(sizeof(double) * ((size_t)n * N + 1));
        double* tmp = (double*)malloc(sizeof(double) * 5 * (size_t)N);
        for (int r = 0; r < n; ++r) {
            orc_orbitals(p, s, R + 3 * (off + r), tmp);
            memcpy(rows + (size_t)r * N, tmp, sizeof(double) * N);
        }
        double* drow = NULL;
        if (s == se) {
            orc_orbitals(p, s, R + 3 * elec, tmp);
            drow = tmp + N; /* channels 1..4 */
            ld = (double*)malloc(sizeof(double) * 4 * (size_t)ne);
            sgd = (double*)malloc(sizeof(double) * 4 * (size_t)ne);
        }
        l[s] = (double*)malloc(sizeof(double) * ne);
        sg[s] = (double*)malloc(sizeof(double) * ne);
        spin_logdets(p, s, rows, ie, drow, l[s], sg[s], s == se ? ld : NULL, s == se ? sgd : NULL);
        free(rows);
        free(tmp);
    }
    /* common scale: the largest |det_up det_dn| over the terms */
    double Lmax = -INFINITY;
    for (int64_t I = 0; I < p->n_det; ++I) {
        double v = l[0][p->det_up[I]] + l[1][p->det_dn[I]];
        if (v > Lmax) Lmax = v;
    }
    double S = 0.0, G[4] = {0, 0, 0, 0}, aS = 0.0, aG[4] = {0, 0, 0, 0};
    if (Lmax > -INFINITY) {
        for (int64_t I = 0; I < p->n_det; ++I) {
            const int u = p->det_up[I], d = p->det_dn[I];
            const double term = p->ci[I] * sg[0][u] * sg[1][d] * exp(l[0][u] + l[1][d] - Lmax);
            S += term;
            aS += fabs(term);
            if (se >= 0) {
                const int us = se ? d : u, uo = se ? u : d;
                const int so = 1 - se;
                const int ne = p->n_exc[se];
                for (int a = 0; a < 4; ++a) {
                    const double t = p->ci[I] * sgd[(size_t)a * ne + us] * sg[so][uo] *
                                     exp(ld[(size_t)a * ne + us] + l[so][uo] - Lmax);
                    G[a] += t;
                    aG[a] += fabs(t);
                }
            }
        }
    }
    int ret = 0;
    if (S == 0.0) {
        *logabs = -INFINITY;
        *sign = 0.0;
        ret = 1;
    } else {
        *logabs = Lmax + log(fabs(S));
        *sign = S > 0 ? 1.0 : -1.0;
    }
    if (se >= 0) {
        if (grad) for (int a = 0; a < 3; ++a) grad[a] = G[a] / S;
        if (lap) lap[0] = G[3] / S;
    }
    if (absum) {
        absum[0] = aS / fabs(S);
        for (int a = 0; a < 4; ++a) absum[1 + a] = aG[a] / fabs(S);
    }
    for (int s = 0; s < 2; ++s) { free(l[s]); free(sg[s]); }
    free(ld);
    free(sgd);
    return ret;
}

/* Per walker w: configuration R[w] with electron elec moved to rnew[w] (if rnew != NULL),
 * evaluated by orc_eval.  Arrays: R [W][n_tot][3], rnew [W][3], grad [W][3], absum [W][5]. */
void orc_eval_batch(const orc_problem* p, int W, const double* R, int elec, const double* rnew,
                    double* logabs, double* sign, double* grad, double* lap, double* absum) {
    const int nt = p->n_elec[0] + p->n_elec[1];
    const int outer = W >= 2 * orc_num_threads();
#pragma omp parallel for schedule(dynamic, 1) if (outer)
    for (int w = 0; w < W; ++w) {
        double* Rw = (double*)malloc(sizeof(double) * 3 * (size_t)nt);
        memcpy(Rw, R + (size_t)w * 3 * nt, sizeof(double) * 3 * nt);
        if (rnew && elec >= 0)
            for (int a = 0; a < 3; ++a) Rw[3 * elec + a] = rnew[3 * w + a];
        orc_eval(p, Rw, elec, &logabs[w], &sign[w], grad ? grad + 3 * w : NULL, lap ? lap + w : NULL,
                 absum ? absum + 5 * w : NULL);
        free(Rw);
    }
}

/*
 * Derivatives of log|Psi| at R with respect to the CI coefficients and the orbital
 * coefficients.  Psi is linear in c, so d log|Psi| / d c_I = det_up,I det_dn,I / Psi.
 * Through M_s,I(r, c) = sum_mu chi_mu(r_r) B_s[mu][col(c)] and Jacobi's formula
 * d det M / d M(r, c) = det M (M^{-1})(c, r):
 *   d log|Psi| / d B_s[mu][j] = sum_I c_I det M_other,I sum_{r, c: col(c) = j}
 *                               chi_mu(r_r) det M_s,I (M_s,I^{-1})(c, r) / Psi.
 * dci [n_det]; dB[s] [n_basis][n_orb[s]] (per spin; a restricted B gets their sum).
 * dB_scale[s] (optional, same shape): the same double sum with every term replaced by its
 * absolute value, |c_I det M_other,I| |chi_mu(r_r)| |det M_s,I (M_s,I^{-1})(c, r)| / |Psi|:
 * the size of the terms that cancel in dB[s], against which its rounding is judged.
 */
int orc_dlogpsi(const orc_problem* p, const double* R, double* dci, double* dB0, double* dB1, double* dB0_scale,
                double* dB1_scale) {
    double* dB[2] = {dB0, dB1};
    double* dBs[2] = {dB0_scale, dB1_scale};
    const int nb = p->n_basis;
    double* l[2];
    double* sg[2];
    double* rows[2];
    double* chi_rows[2];
    for (int s = 0; s < 2; ++s) {
        const int n = p->n_elec[s], N = p->n_orb[s], ne = p->n_exc[s];
        const int off = s ? p->n_elec[0] : 0;
        rows[s] = (double*)malloc(sizeof(double) * ((size_t)n * N + 1));
        chi_rows[s] = (double*)malloc(sizeof(double) * ((size_t)n * nb + 1));
        double* tmp = (double*)malloc(sizeof(double) * 5 * (size_t)N);
        double* chi = (double*)malloc(sizeof(double) * 5 * (size_t)nb);
        for (int r = 0; r < n; ++r) {
            orc_orbitals(p, s, R + 3 * (off + r), tmp);
            memcpy(rows[s] + (size_t)r * N, tmp, sizeof(double) * N);
            orc_basis(p, R + 3 * (off + r), chi);
            memcpy(chi_rows[s] + (size_t)r * nb, chi, sizeof(double) * nb);
        }
        free(tmp);
        free(chi);
        l[s] = (double*)malloc(sizeof(double) * ne);
        sg[s] = (double*)malloc(sizeof(double) * ne);
        spin_logdets(p, s, rows[s], -1, NULL, l[s], sg[s], NULL, NULL);
    }
    double Lmax = -INFINITY;
    for (int64_t I = 0; I < p->n_det; ++I) {
        double v = l[0][p->det_up[I]] + l[1][p->det_dn[I]];
        if (v > Lmax) Lmax = v;
    }
    double S = 0.0;
    for (int64_t I = 0; I < p->n_det; ++I) {
        const int u = p->det_up[I], d = p->det_dn[I];
        S += p->ci[I] * sg[0][u] * sg[1][d] * exp(l[0][u] + l[1][d] - Lmax);
    }
    if (S == 0.0) return 1;
    for (int64_t I = 0; I < p->n_det; ++I) {
        const int u = p->det_up[I], d = p->det_dn[I];
        dci[I] = sg[0][u] * sg[1][d] * exp(l[0][u] + l[1][d] - Lmax) / S;
    }
    /* weight of each string of spin s: W_s[u] = sum_{I: s-string u} c_I det_other / (Psi / det-scale) */
    for (int s = 0; s < 2; ++s) {
        const int n = p->n_elec[s], N = p->n_orb[s], ne = p->n_exc[s];
        const int so = 1 - s;
        double* wgt = (double*)calloc((size_t)ne, sizeof(double));
        double* wabs = (double*)calloc((size_t)ne, sizeof(double));
        double Ls = -INFINITY;
        for (int u = 0; u < ne; ++u) if (l[s][u] > Ls) Ls = l[s][u];
        for (int64_t I = 0; I < p->n_det; ++I) {
            const int us = s ? p->det_dn[I] : p->det_up[I];
            const int uo = s ? p->det_up[I] : p->det_dn[I];
            wgt[us] += p->ci[I] * sg[so][uo] * exp(l[so][uo] + Ls - Lmax);
            wabs[us] += fabs(p->ci[I]) * exp(l[so][uo] + Ls - Lmax);
        }
        /* phibar[r][j] = sum_u wgt[u] sum_{c: col_u(c) = j} cof_u(r, c) e^{-Ls} / S */
        double* phibar = (double*)calloc((size_t)n * N + 1, sizeof(double));
        /* the same sum with every term by its absolute value: the cancellation scale of phibar */
        double* phiabs = (double*)calloc((size_t)n * N + 1, sizeof(double));
#pragma omp parallel
        {
            double* A = (double*)malloc(sizeof(double) * ((size_t)n * n + 1));
            double* lu = (double*)malloc(sizeof(double) * ((size_t)n * n + 1));
            double* inv = (double*)malloc(sizeof(double) * ((size_t)n * n + 1));
            double* col = (double*)malloc(sizeof(double) * ((size_t)n + 1));
            int* perm = (int*)malloc(sizeof(int) * ((size_t)n + 1));
            int* cols = (int*)malloc(sizeof(int) * ((size_t)n + 1));
            double* loc = (double*)calloc((size_t)n * N + 1, sizeof(double));
            double* lab = (double*)calloc((size_t)n * N + 1, sizeof(double));
#pragma omp for schedule(dynamic, 16)
            for (int u = 0; u < ne; ++u) {
                if (wabs[u] == 0.0 || sg[s][u] == 0.0) continue;
                string_columns(p, s, u, cols);
                for (int r = 0; r < n; ++r)
                    for (int c = 0; c < n; ++c) A[(size_t)r * n + c] = rows[s][(size_t)r * N + cols[c]];
                if (lu_inverse(n, A, lu, perm, inv, col)) continue;
                const double detw = wgt[u] * sg[s][u] * exp(l[s][u] - Ls) / S;
                const double deta = wabs[u] * exp(l[s][u] - Ls) / fabs(S);
                for (int r = 0; r < n; ++r)
                    for (int c = 0; c < n; ++c) {
                        loc[(size_t)r * N + cols[c]] += detw * inv[(size_t)c * n + r];
                        lab[(size_t)r * N + cols[c]] += deta * fabs(inv[(size_t)c * n + r]);
                    }
            }
#pragma omp critical
            for (size_t q = 0; q < (size_t)n * N; ++q) {
                phibar[q] += loc[q];
                phiabs[q] += lab[q];
            }
            free(A); free(lu); free(inv); free(col); free(perm); free(cols); free(loc); free(lab);
        }
        for (int mu = 0; mu < nb; ++mu)
            for (int j = 0; j < N; ++j) {
                double acc = 0.0;
                for (int r = 0; r < n; ++r) acc += chi_rows[s][(size_t)r * nb + mu] * phibar[(size_t)r * N + j];
                dB[s][(size_t)mu * N + j] = acc;
                if (dBs[s]) {
                    double sa = 0.0;
                    for (int r = 0; r < n; ++r)
                        sa += fabs(chi_rows[s][(size_t)r * nb + mu]) * phiabs[(size_t)r * N + j];
                    dBs[s][(size_t)mu * N + j] = sa;
                }
            }
        free(wgt);
        free(wabs);
        free(phibar);
        free(phiabs);
    }
    for (int s = 0; s < 2; ++s) { free(l[s]); free(sg[s]); free(rows[s]); free(chi_rows[s]); }
    return 0;
}
