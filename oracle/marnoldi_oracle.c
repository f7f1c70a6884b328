/*
 * Plain, slow FP64 CPU oracle of the multiple Arnoldi (mArnoldi) method.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this library; the product library never does, and the
 * two share no code.
 *
 * Method (Hoshi, Yamazaki, Akiyama, arXiv:1307.3218, Section 2, Eq. 1 and the
 * paragraph after Eq. 2): instead of the generalized eigenproblem
 * H phi = eps S phi (Eq. 2), solve the shifted equations (z S - H) x = e_j
 * (Eq. 1) for every basis index j inside a nu-dimensional Krylov subspace
 * L_nu^(j) that contains e_j.  Each subspace gives a small nu x nu *standard*
 * eigenproblem, whose levels eps_a and vectors v_a determine the Green's
 * function column, hence the density matrix and the energy.
 *
 * Readings of points the paper leaves open (the same readings the library
 * documents):
 *   - L_nu^(j) = span{e_j, H e_j, ..., H^(nu-1) e_j} with an S-orthonormal basis
 *     K = [k_1..k_nu] (K^T S K = I), so that the subspace problem is standard;
 *   - k_1 = e_j / sqrt(S_jj);
 *   - orthogonalisation: modified Gram-Schmidt in the S inner product, two
 *     passes, using the stored vectors S k_i;
 *   - breakdown: stop when beta = ||w||_S <= tau ||u||_S, u = H k_n, record nu_eff;
 *   - subspace matrix: the explicit H_sub = K^T H K, symmetrised as (A + A^T)/2;
 *   - the subspace eigenproblem is solved here by cyclic Jacobi rotations
 *     (a different algorithm from the library's Householder + QL);
 *   - q = K^T e_j, t = V^T q, weight w_a = sqrt(S_jj) V[0][a] t_a;
 *   - Green's function column G(z) e_j = K V diag(1/(z - eps)) t, density
 *     column rho e_j = K V diag(2 f) t, energy-density column
 *     rho^E e_j = K V diag(2 f eps) t with f(x) = 1 / (1 + e^x) at
 *     x = (eps - mu) / kT (spin factor 2);
 *   - electron count N(mu) = sum_j sum_a 2 f w_a and band energy
 *     E = sum_j sum_a 2 f eps_a w_a; mu by bisection on N(mu) = N_e.
 *
 * BSR layout of H and S: row_ptr[n_block_rows + 1] (int64), col_idx[nnzb]
 * (int32), vals[nnzb][4][4] row-major; orbital index 4 I + a.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* y = A x for a BSR matrix with 4x4 row-major blocks. */
static void bsr_apply(int64_t nbr, const int64_t *rp, const int32_t *ci, const double *vals,
                      const double *x, double *y)
{
    for (int64_t I = 0; I < nbr; ++I) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
            const double *B = vals + 16 * k;
            const double *xj = x + 4 * (int64_t)ci[k];
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b)
                    acc[a] += B[4 * a + b] * xj[b];
        }
        for (int a = 0; a < 4; ++a) y[4 * I + a] = acc[a];
    }
}

static double dot(int64_t m, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t r = 0; r < m; ++r) s += a[r] * b[r];
    return s;
}

/* Diagonal element S_jj read from the diagonal block of block-row j/4. */
static double diag_elem(const int64_t *rp, const int32_t *ci, const double *vals, int64_t j)
{
    int64_t J = j / 4;
    int b = (int)(j % 4);
    for (int64_t k = rp[J]; k < rp[J + 1]; ++k)
        if (ci[k] == (int32_t)J) return vals[16 * k + 4 * b + b];
    return 0.0;
}

/*
 * Cyclic Jacobi eigensolver for a symmetric n x n matrix A (row-major, destroyed).
 * On return eps[0..n) ascending and V (row-major, V[i*n + a] = component i of
 * eigenvector a) orthonormal.  Returns the number of sweeps, or -1 if it did not
 * converge in 100 sweeps.
 */
int oracle_jacobi_eigh(int n, double *A, double *eps, double *V)
{
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < n; ++a) V[i * n + a] = (i == a) ? 1.0 : 0.0;
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int p = 0; p < n; ++p) {
            dg += A[p * n + p] * A[p * n + p];
            for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
        }
        if (off <= 1e-34 * (dg + off) || off == 0.0) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double tn = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(tn * tn + 1.0);
                double s = tn * c;
                /* A <- A J (columns p, q), then A <- J^T A (rows p, q), V <- V J. */
                for (int r = 0; r < n; ++r) {
                    double arp = A[r * n + p], arq = A[r * n + q];
                    A[r * n + p] = c * arp - s * arq;
                    A[r * n + q] = s * arp + c * arq;
                }
                for (int r = 0; r < n; ++r) {
                    double apr = A[p * n + r], aqr = A[q * n + r];
                    A[p * n + r] = c * apr - s * aqr;
                    A[q * n + r] = s * apr + c * aqr;
                }
                A[p * n + q] = 0.0;
                A[q * n + p] = 0.0;
                for (int r = 0; r < n; ++r) {
                    double vrp = V[r * n + p], vrq = V[r * n + q];
                    V[r * n + p] = c * vrp - s * vrq;
                    V[r * n + q] = s * vrp + c * vrq;
                }
            }
        }
    }
    for (int a = 0; a < n; ++a) eps[a] = A[a * n + a];
    /* ascending order: selection sort of levels with their vectors */
    for (int a = 0; a < n; ++a) {
        int best = a;
        for (int b = a + 1; b < n; ++b)
            if (eps[b] < eps[best]) best = b;
        if (best != a) {
            double e = eps[a]; eps[a] = eps[best]; eps[best] = e;
            for (int r = 0; r < n; ++r) {
                double v = V[r * n + a]; V[r * n + a] = V[r * n + best]; V[r * n + best] = v;
            }
        }
    }
    return sweep < 100 ? sweep : -1;
}

/*
 * One column j (global mode: vectors over all M = 4 nbr orbitals).
 *
 * Outputs (nu entries each; entries a >= nu_eff are zero):
 *   eps[a] subspace levels ascending, w[a] weights, t[a] = (V^T q)_a;
 *   Y[r*nu + a] = (K V)[rows[r]][a] for the nrows requested rows;
 *   Hsub (nu*nu, may be NULL) the symmetrised subspace matrix (nu_eff x nu_eff block);
 *   Kout (nu*M, may be NULL) the basis, Kout[i*M + r] = k_i[r].
 * Returns nu_eff (>= 1), or a negative value on allocation or eigensolver failure.
 */
int oracle_column(int64_t nbr, const int64_t *rp, const int32_t *ci, const double *Hv,
                  const double *Sv, int64_t j, int nu, double tau, int64_t nrows,
                  const int64_t *rows, double *eps, double *w, double *t, double *Y,
                  double *Hsub, double *Kout)
{
    const int64_t m = 4 * nbr;
    double *K = (double *)calloc((size_t)m * nu, sizeof(double));
    double *SK = (double *)calloc((size_t)m * nu, sizeof(double));
    double *u = (double *)malloc(sizeof(double) * m);
    double *wv = (double *)malloc(sizeof(double) * m);
    double *Sw = (double *)malloc(sizeof(double) * m);
    double *Su = (double *)malloc(sizeof(double) * m);
    double *A = (double *)malloc(sizeof(double) * nu * nu);
    double *V = (double *)malloc(sizeof(double) * nu * nu);
    double *ev = (double *)malloc(sizeof(double) * nu);
    int nu_eff = nu, rc = 0;
    if (!K || !SK || !u || !wv || !Sw || !Su || !A || !V || !ev) { rc = -2; goto done; }

    /* k_1 = e_j / sqrt(S_jj), S k_1 by an explicit product. */
    const double sjj = diag_elem(rp, ci, Sv, j);
    if (!(sjj > 0.0)) { rc = -3; goto done; }
    K[j] = 1.0 / sqrt(sjj);
    bsr_apply(nbr, rp, ci, Sv, K, SK);

    for (int n = 0; n + 1 < nu; ++n) {
        const double *kn = K + (int64_t)n * m;
        bsr_apply(nbr, rp, ci, Hv, kn, u);               /* u = H k_n */
        memcpy(wv, u, sizeof(double) * m);
        for (int pass = 0; pass < 2; ++pass) {            /* MGS in the S inner product, twice */
            for (int i = 0; i <= n; ++i) {
                const double *ki = K + (int64_t)i * m, *ski = SK + (int64_t)i * m;
                double c = dot(m, ski, wv);
                for (int64_t r = 0; r < m; ++r) wv[r] -= c * ki[r];
            }
        }
        bsr_apply(nbr, rp, ci, Sv, wv, Sw);               /* S w */
        double beta2 = dot(m, wv, Sw);
        bsr_apply(nbr, rp, ci, Sv, u, Su);                /* S u, for the breakdown test */
        const double unorm2 = dot(m, u, Su);
        if (!(beta2 > 0.0) || sqrt(beta2) <= tau * sqrt(unorm2)) { nu_eff = n + 1; break; }
        const double beta = sqrt(beta2);
        double *kn1 = K + (int64_t)(n + 1) * m, *skn1 = SK + (int64_t)(n + 1) * m;
        for (int64_t r = 0; r < m; ++r) { kn1[r] = wv[r] / beta; skn1[r] = Sw[r] / beta; }
    }

    /* H_sub = K^T H K over the nu_eff basis vectors, symmetrised. */
    {
        const int ne = nu_eff;
        double *HK = (double *)malloc(sizeof(double) * m * ne);
        if (!HK) { rc = -2; goto done; }
        for (int l = 0; l < ne; ++l) bsr_apply(nbr, rp, ci, Hv, K + (int64_t)l * m, HK + (int64_t)l * m);
        for (int i = 0; i < ne; ++i)
            for (int l = 0; l < ne; ++l) A[i * ne + l] = dot(m, K + (int64_t)i * m, HK + (int64_t)l * m);
        free(HK);
        for (int i = 0; i < ne; ++i)
            for (int l = i + 1; l < ne; ++l) {
                double s = 0.5 * (A[i * ne + l] + A[l * ne + i]);
                A[i * ne + l] = s;
                A[l * ne + i] = s;
            }
        if (Hsub) {
            for (int i = 0; i < nu * nu; ++i) Hsub[i] = 0.0;
            for (int i = 0; i < ne; ++i)
                for (int l = 0; l < ne; ++l) Hsub[i * nu + l] = A[i * ne + l];
        }
        if (oracle_jacobi_eigh(ne, A, ev, V) < 0) { rc = -4; goto done; }

        /* q = K^T e_j (row j of K), t = V^T q, w_a = sqrt(S_jj) V[0][a] t_a. */
        for (int a = 0; a < nu; ++a) { eps[a] = 0.0; w[a] = 0.0; t[a] = 0.0; }
        for (int a = 0; a < ne; ++a) {
            double ta = 0.0;
            for (int i = 0; i < ne; ++i) ta += V[i * ne + a] * K[(int64_t)i * m + j];
            eps[a] = ev[a];
            t[a] = ta;
            w[a] = sqrt(sjj) * V[0 * ne + a] * ta;
        }
        /* Y = (K V) restricted to the requested rows. */
        for (int64_t rr = 0; rr < nrows; ++rr) {
            const int64_t r = rows[rr];
            for (int a = 0; a < nu; ++a) {
                double s = 0.0;
                if (a < ne)
                    for (int i = 0; i < ne; ++i) s += K[(int64_t)i * m + r] * V[i * ne + a];
                Y[rr * nu + a] = s;
            }
        }
        if (Kout) memcpy(Kout, K, sizeof(double) * m * nu);
    }
    rc = nu_eff;
done:
    free(K); free(SK); free(u); free(wv); free(Sw); free(Su); free(A); free(V); free(ev);
    return rc;
}

/*
 * Many columns, OpenMP over columns only.  Column c writes its nu-vectors at
 * c*nu and its rows rows[row_off[c] .. row_off[c+1]) of K V at Y + row_off[c]*nu.
 * nu_eff[c] receives the per-column status (>= 1 ok, < 0 failure).
 * Returns 0 if every column succeeded, else the first negative status.
 */
int oracle_columns(int64_t nbr, const int64_t *rp, const int32_t *ci, const double *Hv,
                   const double *Sv, int64_t ncols, const int64_t *cols, int nu, double tau,
                   const int64_t *row_off, const int64_t *rows, int *nu_eff, double *eps,
                   double *w, double *t, double *Y, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < ncols; ++c) {
        int r = oracle_column(nbr, rp, ci, Hv, Sv, cols[c], nu, tau, row_off[c + 1] - row_off[c],
                              rows + row_off[c], eps + c * nu, w + c * nu, t + c * nu,
                              Y + row_off[c] * nu, NULL, NULL);
        nu_eff[c] = r;
        if (r < 0) {
#pragma omp critical
            if (bad == 0) bad = r;
        }
    }
    return bad;
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Fermi function f(x) = 1 / (1 + e^x), evaluated through e^{-|x|} so it never overflows. */
double oracle_fermi(double x)
{
    if (x >= 0.0) {
        double e = exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(x));
}

/* N(mu) = sum 2 f((eps-mu)/kT) w and E(mu) = sum 2 f eps w over n stored levels. */
void oracle_count(int64_t n, const double *eps, const double *w, double mu, double kT,
                  double *N, double *E)
{
    double sn = 0.0, se = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double f2 = 2.0 * oracle_fermi((eps[i] - mu) / kT);
        sn += f2 * w[i];
        se += f2 * eps[i] * w[i];
    }
    *N = sn;
    *E = se;
}

/*
 * Bisection for N(mu) = Ne on the bracket [min eps - 40 kT, max eps + 40 kT]:
 * stop when |N - Ne| <= rtol * Ne or after maxit halvings.  Returns the number
 * of evaluations, or -1 if the bracket does not contain Ne.
 */
int oracle_bisect(int64_t n, const double *eps, const double *w, double Ne, double kT,
                  double rtol, int maxit, double *mu_out, double *N_out, double *E_out)
{
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        if (eps[i] < lo) lo = eps[i];
        if (eps[i] > hi) hi = eps[i];
    }
    lo -= 40.0 * kT;
    hi += 40.0 * kT;
    double Nlo, Nhi, E;
    oracle_count(n, eps, w, lo, kT, &Nlo, &E);
    oracle_count(n, eps, w, hi, kT, &Nhi, &E);
    if (!(Nlo <= Ne && Ne <= Nhi)) return -1;
    double mu = 0.5 * (lo + hi), N = 0.0;
    int it;
    for (it = 1; it <= maxit; ++it) {
        mu = 0.5 * (lo + hi);
        oracle_count(n, eps, w, mu, kT, &N, &E);
        if (fabs(N - Ne) <= rtol * Ne) break;
        if (N < Ne) lo = mu; else hi = mu;
    }
    *mu_out = mu;
    *N_out = N;
    *E_out = E;
    return it;
}

/*
 * Density and energy-density values from stored column data:
 * rho[r] = sum_a Y[r][a] 2 f_a t_a, rhoE[r] = sum_a Y[r][a] 2 f_a eps_a t_a, for the
 * rows of each column (layout as in oracle_columns).
 */
void oracle_density(int64_t ncols, int nu, const int64_t *row_off, const double *eps,
                    const double *t, const double *Y, double mu, double kT, double *rho,
                    double *rhoE)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < ncols; ++c) {
        double y[1024], ye[1024];
        int nn = nu < 1024 ? nu : 1024;
        for (int a = 0; a < nn; ++a) {
            double f2 = 2.0 * oracle_fermi((eps[c * nu + a] - mu) / kT);
            y[a] = f2 * t[c * nu + a];
            ye[a] = f2 * eps[c * nu + a] * t[c * nu + a];
        }
        for (int64_t r = row_off[c]; r < row_off[c + 1]; ++r) {
            double s = 0.0, se = 0.0;
            for (int a = 0; a < nn; ++a) {
                s += Y[r * nu + a] * y[a];
                se += Y[r * nu + a] * ye[a];
            }
            rho[r] = s;
            rhoE[r] = se;
        }
    }
}
