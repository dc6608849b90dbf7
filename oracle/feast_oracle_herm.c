/*
 * feast_oracle_herm.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain FP64 CPU FEAST for complex Hermitian sparse problems A x = lambda B x
 * (A Hermitian, B Hermitian positive definite; the guide's zfeast_hcsr{ev,gv},
 * Sec. 3.2 "FEAST Hermitian").  Same role and rules as feast_oracle.c: it
 * checks the library, shares no code with it, and is only called from tests.
 *
 * What changes from the real symmetric case:
 *   - The spectral projector's lower half contour is no longer the complex
 *     conjugate of the upper half.  With G(z) = (zB - A)^{-1} and real
 *     eigenvalues, G(z)B = sum_i x_i x_i^H B / (z - lambda_i), so the filter
 *     rho(lambda) = sum_e Re(w_e / (z_e - lambda))
 *                 = sum_e (1/2)[w_e/(z_e - lambda) + conj(w_e)/(conj(z_e) - lambda)]
 *     is applied to a block by Q = sum_e (1/2)[w_e G(z_e) + conj(w_e) G(conj z_e)] B Y:
 *     two shifted solves per node, at z_e and at its conjugate.
 *   - zB - A is not complex symmetric, so the direct solver is a banded LU
 *     without pivoting.  It exists and is stable because -i(zB - A) (Im z > 0)
 *     and i(zB - A) (Im z < 0) have the positive definite Hermitian part
 *     |Im z| B.
 *   - Rayleigh-Ritz uses Q^H A Q and Q^H B Q, symmetrised as (M + M^H)/2, and a
 *     Hermitian Jacobi: the phase e = a_pq/|a_pq| is taken out by
 *     D = diag(1, conj(e)) on (p, q), leaving the real symmetric rotation.
 * Blocks are column-major n x m arrays of double complex ((re, im) pairs).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

int orc_contour_gauss(int ne, double emin, double emax, double ratio, double* z, double* w);
int orc_contour_trapezoid(int ne, double emin, double emax, double ratio, double* z, double* w);
int orc_contour_zolotarev(int ne, double emin, double emax, double eta, double* z, double* w);

typedef struct {
    int n;
    const int* ip;
    const int* ix;
    const cplx* v;
} hcsr;

static void h_mm(const hcsr* A, int m, const cplx* X, cplx* Y)
{
    const int n = A->n;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < n; ++i) {
            cplx s = 0.0;
            for (int p = A->ip[i]; p < A->ip[i + 1]; ++p) s += A->v[p] * X[(size_t)j * n + A->ix[p]];
            Y[(size_t)j * n + i] = s;
        }
}

static void hb_mm(const hcsr* B, int n, int m, const cplx* X, cplx* Y)
{
    if (B) h_mm(B, m, X, Y);
    else memcpy(Y, X, sizeof(cplx) * (size_t)n * m);
}

void orc_h_csr_mm(int n, const int* ip, const int* ix, const cplx* v, int m, const cplx* X, cplx* Y)
{
    hcsr A = {n, ip, ix, v};
    h_mm(&A, m, X, Y);
}

/* ------------------------------------------------------------------------ */
/* Banded LU without pivoting of K = zB - A: band[i*ld + (j - i + bw)] holds
 * K_ij for |i - j| <= bw, ld = 2 bw + 1; on return the unit lower factor L
 * (below the diagonal) and U (diagonal and above) in the same places. */
static int h_bandwidth(const hcsr* A)
{
    int bw = 0;
    for (int i = 0; i < A->n; ++i)
        for (int p = A->ip[i]; p < A->ip[i + 1]; ++p) {
            int d = abs(i - A->ix[p]);
            if (d > bw) bw = d;
        }
    return bw;
}

#define BAND(i, j) band[(size_t)(i) * ld + ((j) - (i) + bw)]

static int band_lu(int n, int bw, cplx* band)
{
    const int ld = 2 * bw + 1;
    for (int k = 0; k < n; ++k) {
        cplx piv = BAND(k, k);
        if (cabs(piv) == 0.0) return -1;
        int i1 = k + bw < n - 1 ? k + bw : n - 1;
        for (int i = k + 1; i <= i1; ++i) {
            cplx l = BAND(i, k) / piv;
            BAND(i, k) = l;
            for (int j = k + 1; j <= i1; ++j) BAND(i, j) -= l * BAND(k, j);
        }
    }
    return 0;
}

static void band_lu_solve(int n, int bw, const cplx* band, cplx* x)
{
    const int ld = 2 * bw + 1;
    for (int i = 0; i < n; ++i) { /* L y = b */
        cplx s = x[i];
        int k0 = i - bw < 0 ? 0 : i - bw;
        for (int k = k0; k < i; ++k) s -= BAND(i, k) * x[k];
        x[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) { /* U x = y */
        cplx s = x[i];
        int k1 = i + bw < n - 1 ? i + bw : n - 1;
        for (int k = i + 1; k <= k1; ++k) s -= BAND(i, k) * x[k];
        x[i] = s / BAND(i, i);
    }
}

/* (z B - A) X = R for the m columns of R (column-major n x m).  Returns 0 or -2. */
static int h_shifted_solve(const hcsr* A, const hcsr* B, cplx z, int m, const cplx* R, cplx* X)
{
    const int n = A->n;
    int bw = h_bandwidth(A);
    if (B) {
        int bb = h_bandwidth(B);
        if (bb > bw) bw = bb;
    }
    const int ld = 2 * bw + 1;
    cplx* band = (cplx*)calloc((size_t)n * ld, sizeof(cplx));
    if (!band) return -2;
    for (int i = 0; i < n; ++i) {
        for (int p = A->ip[i]; p < A->ip[i + 1]; ++p) BAND(i, A->ix[p]) -= A->v[p];
        if (B)
            for (int p = B->ip[i]; p < B->ip[i + 1]; ++p) BAND(i, B->ix[p]) += z * B->v[p];
        else
            BAND(i, i) += z;
    }
    int st = band_lu(n, bw, band);
    if (st == 0) {
        memcpy(X, R, sizeof(cplx) * (size_t)n * m);
#pragma omp parallel for schedule(dynamic)
        for (int j = 0; j < m; ++j) band_lu_solve(n, bw, band, X + (size_t)j * n);
    }
    free(band);
    return st ? -2 : 0;
}
#undef BAND

int orc_h_shifted_solve(int n, const int* ip, const int* ix, const cplx* av, const int* bip, const int* bix,
                        const cplx* bv, double zr, double zi, int m, const cplx* R, cplx* X)
{
    hcsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    return h_shifted_solve(&A, bip ? &Bm : NULL, zr + I * zi, m, R, X);
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi for a Hermitian n x n matrix a (column-major, destroyed):
 * w ascending, V unitary with A V = V diag(w).  Rotation of (p, q): with
 * e = a_pq / |a_pq|, tau = (a_qq - a_pp) / (2 |a_pq|),
 * t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c,
 * J = D R on columns (p, q): J_pp = c, J_pq = s, J_qp = -s conj(e),
 * J_qq = c conj(e), and A <- J^H A J, V <- V J.  Returns 0 or -1. */
int orc_h_jacobi_eig(int n, cplx* a, double* w, cplx* V)
{
#define A_(i, j) a[(size_t)(j) * n + (i)]
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) V[(size_t)j * n + i] = i == j ? 1.0 : 0.0;
    double fro = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) fro += creal(a[k] * conj(a[k]));
    const double absfloor = 1e-18 * sqrt(fro);
    int sweep, rotated = 1;
    for (sweep = 0; sweep < 100 && rotated; ++sweep) {
        rotated = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const cplx apq = A_(p, q);
                const double mag = cabs(apq);
                const double app = creal(A_(p, p)), aqq = creal(A_(q, q));
                const double thr = fmax(1.1e-16 * sqrt(fabs(app * aqq)), absfloor);
                if (!(mag > thr)) continue;
                rotated = 1;
                const cplx e = apq / mag, ec = conj(e);
                const double tau = (aqq - app) / (2.0 * mag);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int i = 0; i < n; ++i) { /* columns: M = A J */
                    const cplx xp = A_(i, p), xq = A_(i, q);
                    A_(i, p) = c * xp - s * ec * xq;
                    A_(i, q) = s * xp + c * ec * xq;
                }
                for (int j = 0; j < n; ++j) { /* rows: J^H M */
                    const cplx yp = A_(p, j), yq = A_(q, j);
                    A_(p, j) = c * yp - s * e * yq;
                    A_(q, j) = s * yp + c * e * yq;
                }
                A_(p, q) = 0.0;
                A_(q, p) = 0.0;
                A_(p, p) = creal(A_(p, p));
                A_(q, q) = creal(A_(q, q));
                for (int i = 0; i < n; ++i) {
                    const cplx vp = V[(size_t)p * n + i], vq = V[(size_t)q * n + i];
                    V[(size_t)p * n + i] = c * vp - s * ec * vq;
                    V[(size_t)q * n + i] = s * vp + c * ec * vq;
                }
            }
    }
    /* ascending order (selection by rank, ties by index) */
    int* rank = (int*)malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) {
        int r = 0;
        for (int j = 0; j < n; ++j) {
            const double li = creal(A_(i, i)), lj = creal(A_(j, j));
            r += (lj < li) || (lj == li && j < i);
        }
        rank[i] = r;
    }
    cplx* Vs = (cplx*)malloc(sizeof(cplx) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        w[rank[i]] = creal(A_(i, i));
        memcpy(Vs + (size_t)rank[i] * n, V + (size_t)i * n, sizeof(cplx) * n);
    }
    memcpy(V, Vs, sizeof(cplx) * (size_t)n * n);
    free(Vs);
    free(rank);
    return sweep >= 100 ? -1 : 0;
#undef A_
}

/* Reduced generalized Hermitian problem Aq v = lambda Bq v (m x m): scale by
 * D = diag(Bq)^{-1/2}; Jacobi on D Bq D = U diag(d) U^H; keep d > 1e-14 max d;
 * S = D U_k d_k^{-1/2}; Jacobi on S^H Aq S = W Lambda W^H; V = S W (m x k,
 * V^H Bq V = I).  Both inputs symmetrised as (M + M^H)/2.  Returns 0 or -3. */
int orc_h_reduced_gev(int m, const cplx* Aq, const cplx* Bq, double* lam, cplx* V, int* mk)
{
    const size_t mm = (size_t)m * m;
    double* dsc = (double*)malloc(sizeof(double) * m);
    cplx* b = (cplx*)malloc(sizeof(cplx) * mm);
    cplx* As = (cplx*)malloc(sizeof(cplx) * mm);
    cplx* U = (cplx*)malloc(sizeof(cplx) * mm);
    double* d = (double*)malloc(sizeof(double) * m);
    int info = 0;
    for (int i = 0; i < m; ++i) {
        const double bii = creal(Bq[(size_t)i * m + i]);
        dsc[i] = bii > 0.0 ? 1.0 / sqrt(bii) : 0.0;
    }
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
            const cplx bs = 0.5 * (Bq[(size_t)j * m + i] + conj(Bq[(size_t)i * m + j]));
            b[(size_t)j * m + i] = bs * dsc[i] * dsc[j];
            As[(size_t)j * m + i] = 0.5 * (Aq[(size_t)j * m + i] + conj(Aq[(size_t)i * m + j]));
        }
    orc_h_jacobi_eig(m, b, d, U);
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) if (d[i] > dmax) dmax = d[i];
    int k = 0;
    if (dmax > 0.0)
        for (int i = 0; i < m; ++i) if (d[i] > 1e-14 * dmax) ++k;
    if (k == 0) { info = -3; *mk = 0; goto out; }
    {
        cplx* S = (cplx*)malloc(sizeof(cplx) * (size_t)m * k);
        int c = 0;
        for (int i = m - 1; i >= 0 && c < k; --i) {
            if (!(d[i] > 1e-14 * dmax)) continue;
            const double sc = 1.0 / sqrt(d[i]);
            for (int r = 0; r < m; ++r) S[(size_t)c * m + r] = dsc[r] * U[(size_t)i * m + r] * sc;
            ++c;
        }
        cplx* AS = (cplx*)malloc(sizeof(cplx) * (size_t)m * k);
        cplx* C = (cplx*)malloc(sizeof(cplx) * (size_t)k * k);
        cplx* W = (cplx*)malloc(sizeof(cplx) * (size_t)k * k);
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < m; ++i) {
                cplx s = 0.0;
                for (int l = 0; l < m; ++l) s += As[(size_t)l * m + i] * S[(size_t)j * m + l];
                AS[(size_t)j * m + i] = s;
            }
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < k; ++i) {
                cplx s = 0.0;
                for (int l = 0; l < m; ++l) s += conj(S[(size_t)i * m + l]) * AS[(size_t)j * m + l];
                C[(size_t)j * k + i] = s;
            }
        for (int j = 0; j < k; ++j) /* Hermitian part before Jacobi */
            for (int i = j; i < k; ++i) {
                const cplx s = 0.5 * (C[(size_t)j * k + i] + conj(C[(size_t)i * k + j]));
                C[(size_t)j * k + i] = s;
                C[(size_t)i * k + j] = conj(s);
            }
        orc_h_jacobi_eig(k, C, lam, W);
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < m; ++i) {
                cplx s = 0.0;
                for (int l = 0; l < k; ++l) s += S[(size_t)l * m + i] * W[(size_t)j * k + l];
                V[(size_t)j * m + i] = s;
            }
        *mk = k;
        free(S); free(AS); free(C); free(W);
    }
out:
    free(dsc); free(b); free(As); free(U); free(d);
    return info;
}

/* ------------------------------------------------------------------------ */
/* Q = sum_e (1/2)[w_e G(z_e) + conj(w_e) G(conj z_e)] B Y, nodes of rule fpm(16).
 * Returns 0 or -2. */
static int h_filter(const hcsr* A, const hcsr* B, int ne, const double* z, const double* w, int m, const cplx* Y,
                    cplx* Q)
{
    const int n = A->n;
    const size_t nm = (size_t)n * m;
    cplx* BY = (cplx*)malloc(sizeof(cplx) * nm);
    cplx* sol = (cplx*)malloc(sizeof(cplx) * nm);
    hb_mm(B, n, m, Y, BY);
    memset(Q, 0, sizeof(cplx) * nm);
    int st = 0;
    for (int e = 0; e < ne && !st; ++e) {
        const cplx ze = z[2 * e] + I * z[2 * e + 1], we = w[2 * e] + I * w[2 * e + 1];
        for (int side = 0; side < 2 && !st; ++side) {
            const cplx zz = side ? conj(ze) : ze, ww = side ? conj(we) : we;
            st = h_shifted_solve(A, B, zz, m, BY, sol);
            if (!st)
                for (size_t k = 0; k < nm; ++k) Q[k] += 0.5 * ww * sol[k];
        }
    }
    free(BY);
    free(sol);
    return st;
}

int orc_h_filter(int n, const int* ip, const int* ix, const cplx* av, const int* bip, const int* bix,
                 const cplx* bv, int ne, double emin, double emax, double ratio, int rule, int m, const cplx* Y,
                 cplx* Q)
{
    hcsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    double* z = (double*)malloc(sizeof(double) * 2 * ne);
    double* w = (double*)malloc(sizeof(double) * 2 * ne);
    if (rule == 2) orc_contour_zolotarev(ne, emin, emax, 0.05, z, w);
    else if (rule == 1) orc_contour_trapezoid(ne, emin, emax, ratio, z, w);
    else orc_contour_gauss(ne, emin, emax, ratio, z, w);
    const int st = h_filter(&A, bip ? &Bm : NULL, ne, z, w, m, Y, Q);
    free(z);
    free(w);
    return st;
}

/* res_j = ||A x_j - lam_j B x_j|| / (alpha ||B x_j||), alpha = max(|emin|,|emax|). */
static void h_residuals(const hcsr* A, const hcsr* B, int m, const cplx* X, const double* lam, double alpha,
                        double* res)
{
    const int n = A->n;
    cplx* AX = (cplx*)malloc(sizeof(cplx) * (size_t)n * m);
    cplx* BX = (cplx*)malloc(sizeof(cplx) * (size_t)n * m);
    h_mm(A, m, X, AX);
    hb_mm(B, n, m, X, BX);
    for (int j = 0; j < m; ++j) {
        double rn = 0.0, bn = 0.0;
        for (int i = 0; i < n; ++i) {
            const cplx r = AX[(size_t)j * n + i] - lam[j] * BX[(size_t)j * n + i];
            rn += creal(r * conj(r));
            bn += creal(BX[(size_t)j * n + i] * conj(BX[(size_t)j * n + i]));
        }
        res[j] = sqrt(rn) / (alpha * sqrt(bn));
    }
    free(AX);
    free(BX);
}

/* FEAST for complex Hermitian CSR problems (zfeast_hcsr{ev,gv} semantics, the
 * classic filter on every loop).  fpm as in orc_feast_scsr (fpm(2) Ne, fpm(3)
 * tolerance, fpm(4) loops, fpm(5) start subspace in X, fpm(16) rule, fpm(18)
 * ratio).  Y0: start block when fpm(5)=0.  On exit E inside ascending then
 * outside ascending, X (n x m0) the matching B-orthonormal Ritz vectors, res,
 * *m0io the kept size.  Returns info (0, 1, 2, 3, -2, -3, 102, 200, 201, 202). */
int orc_feast_hcsr(int n, const int* ip, const int* ix, const cplx* av, const int* bip, const int* bix,
                   const cplx* bv, const int* fpm, double emin, double emax, int* m0io, const cplx* Y0,
                   double* E, cplx* X, double* res, int* Mout, int* loop_out, double* epsout)
{
    const int m0 = *m0io;
    if (n <= 0) return 202;
    if (m0 <= 0 || m0 > n) return 201;
    if (!(emin < emax)) return 200;
    const int ne = fpm[1];
    if (ne < 1) return 102;
    hcsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    const hcsr* B = bip ? &Bm : NULL;
    const double ratio = fpm[17] / 100.0, eps = pow(10.0, -fpm[2]);
    const int maxloop = fpm[3];
    const double alpha = fmax(fabs(emin), fabs(emax));
    double* z = (double*)malloc(sizeof(double) * 2 * ne);
    double* w = (double*)malloc(sizeof(double) * 2 * ne);
    if (fpm[15] == 2) orc_contour_zolotarev(ne, emin, emax, 0.05, z, w);
    else if (fpm[15] == 1) orc_contour_trapezoid(ne, emin, emax, ratio, z, w);
    else orc_contour_gauss(ne, emin, emax, ratio, z, w);
    const size_t nm = (size_t)n * m0;
    cplx* Q = (cplx*)malloc(sizeof(cplx) * nm);
    cplx* AQ = (cplx*)malloc(sizeof(cplx) * nm);
    cplx* BQ = (cplx*)malloc(sizeof(cplx) * nm);
    cplx* Aq = (cplx*)malloc(sizeof(cplx) * m0 * m0);
    cplx* Bq = (cplx*)malloc(sizeof(cplx) * m0 * m0);
    cplx* V = (cplx*)malloc(sizeof(cplx) * m0 * m0);
    double* lam = (double*)malloc(sizeof(double) * m0);
    cplx* Xw = (cplx*)calloc(nm, sizeof(cplx));
    double* rw = (double*)malloc(sizeof(double) * m0);
    int info = 0, k = 0, mk = m0, M = 0;
    double trace_prev = 0.0, eo = 1.0;
    if (h_filter(&A, B, ne, z, w, m0, fpm[4] == 1 ? X : Y0, Q)) { info = -2; goto out; }
    for (k = 0;; ++k) {
        h_mm(&A, mk, Q, AQ);
        hb_mm(B, n, mk, Q, BQ);
#pragma omp parallel for schedule(dynamic)
        for (int j = 0; j < mk; ++j)
            for (int i = 0; i < mk; ++i) {
                cplx sa = 0.0, sb = 0.0;
                for (int r = 0; r < n; ++r) {
                    const cplx q = conj(Q[(size_t)i * n + r]);
                    sa += q * AQ[(size_t)j * n + r];
                    sb += q * BQ[(size_t)j * n + r];
                }
                Aq[(size_t)j * mk + i] = sa;
                Bq[(size_t)j * mk + i] = sb;
            }
        int mk2 = 0;
        if (orc_h_reduced_gev(mk, Aq, Bq, lam, V, &mk2)) { info = -3; goto out; }
#pragma omp parallel for schedule(static)
        for (int j = 0; j < mk2; ++j)
            for (int r = 0; r < n; ++r) {
                cplx s = 0.0;
                for (int l = 0; l < mk; ++l) s += Q[(size_t)l * n + r] * V[(size_t)j * mk + l];
                Xw[(size_t)j * n + r] = s;
            }
        mk = mk2;
        h_residuals(&A, B, mk, Xw, lam, alpha, rw);
        M = 0;
        double trace = 0.0, maxres = 0.0;
        for (int j = 0; j < mk; ++j)
            if (lam[j] >= emin && lam[j] <= emax) {
                ++M;
                trace += lam[j];
                if (rw[j] > maxres) maxres = rw[j];
            }
        eo = k == 0 ? 1.0 : fabs(trace - trace_prev) / alpha;
        trace_prev = trace;
        if (M >= 1 && maxres < eps) { info = 0; break; }
        if (M == 0 && k >= 1) { info = 1; break; }
        if (k >= maxloop) { info = 2; break; }
        if (h_filter(&A, B, ne, z, w, mk, Xw, Q)) { info = -2; goto out; }
    }
    if (info == 0 && M >= mk) info = 3;
    {
        int c = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < mk; ++j) {
                const int in = lam[j] >= emin && lam[j] <= emax;
                if ((pass == 0) != in) continue;
                E[c] = lam[j];
                res[c] = rw[j];
                memcpy(X + (size_t)c * n, Xw + (size_t)j * n, sizeof(cplx) * n);
                ++c;
            }
        for (int j = mk; j < m0; ++j) { E[j] = 0.0; res[j] = 0.0; memset(X + (size_t)j * n, 0, sizeof(cplx) * n); }
    }
out:
    *Mout = M;
    *loop_out = k;
    *epsout = eo;
    *m0io = mk;
    free(z); free(w); free(Q); free(AQ); free(BQ); free(Aq); free(Bq); free(V); free(lam); free(Xw); free(rw);
    return info;
}
