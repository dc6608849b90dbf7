/*
 * feast_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of the FEAST
 * contour-filter eigensolver for real symmetric sparse problems A x = lambda B x
 * (B symmetric positive definite).  It exists to check the CUDA library; it is
 * not part of the product path, shares no code with it, and must only be called
 * from tests/, from __graft_entry__.smoke() and from bench.py's CPU-baseline leg.
 *
 * The FEAST v4.0 guide describes the method in prose (Sec. 1.1 "The FEAST
 * Algorithm", the fpm table of Sec. 3.1, the argument table of Sec. 3.2 and the
 * tips on residual inverse iteration in Sec. 3.1).  It prints no formulas, so
 * the steps below are written from the mathematics the guide refers to:
 *   - the spectral projector P = (1/2 pi i) \oint (zB - A)^{-1} B dz over an
 *     ellipse through Emin/Emax (fpm(18) = ratio), symmetric about the real axis,
 *     so only the upper half contour is integrated (guide Sec. 4.2, "Search
 *     contour");
 *   - Gauss-Legendre quadrature on that half contour (fpm(16)=0);
 *   - Rayleigh-Ritz on Q = P_quad Y, a dense reduced generalized eigenproblem,
 *     Ritz vectors X = Q V and residuals ||A x - lambda B x|| / ||alpha B x||,
 *     alpha = max(|Emin|,|Emax|) (guide Sec. 3.2, argument `res`);
 *   - stop when the largest residual of the pairs inside [Emin,Emax] is below
 *     10^-fpm(3) (fpm(6)=1).
 * Shifted solves are either a banded complex-symmetric LDL^T (no pivoting; the
 * imaginary part Im(z) B is positive definite for Im z > 0) or an FP64 COCG run
 * to a tight tolerance.  Where a function has no independent pin it says so;
 * every other function is pinned by tests/test_oracle.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int n;
    const int* ip;    /* [n+1], 0-based */
    const int* ix;    /* [nnz] */
    const double* v;  /* [nnz] */
} ocsr;

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1,1]: Newton iteration on the Legendre polynomial
 * P_n using the three-term recurrence (k+1)P_{k+1} = (2k+1) x P_k - k P_{k-1};
 * weights 2 / ((1-x^2) P_n'(x)^2).  Nodes returned in descending order.      */
int orc_gauss_legendre(int n, double* x, double* w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = t; p0 = 1.0; }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        {   /* recompute derivative at the converged node */
            double p0 = 1.0, p1 = t;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = t; p0 = 1.0; }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
    return 0;
}

/* Half-contour nodes and weights (Gauss, fpm(16)=0).  With c = (Emin+Emax)/2,
 * r = (Emax-Emin)/2 and a = fpm(18)/100 the upper half ellipse is
 * z(theta) = c + r cos(theta) + i a r sin(theta), theta in [0, pi].  The
 * projector's real part equals (1/pi) Im \int_0^pi f(z) z'(theta) d theta, and
 * Gauss-Legendre in theta = (pi/2)(1 - x) turns it into
 * sum_e Re(w_e f(z_e)) with w_e = omega_e z'(theta_e) / (2i)
 *                               = (omega_e r / 2)(a cos theta_e + i sin theta_e).
 * Output arrays are interleaved (re, im). */
int orc_contour_gauss(int ne, double emin, double emax, double ratio, double* z, double* w)
{
    double* x = (double*)malloc(sizeof(double) * ne);
    double* om = (double*)malloc(sizeof(double) * ne);
    if (orc_gauss_legendre(ne, x, om)) { free(x); free(om); return -1; }
    double c = 0.5 * (emin + emax), r = 0.5 * (emax - emin);
    for (int e = 0; e < ne; ++e) {
        double th = 0.5 * M_PI * (1.0 - x[e]);
        z[2 * e] = c + r * cos(th);
        z[2 * e + 1] = ratio * r * sin(th);
        w[2 * e] = 0.5 * om[e] * r * ratio * cos(th);
        w[2 * e + 1] = 0.5 * om[e] * r * sin(th);
    }
    free(x);
    free(om);
    return 0;
}

/* Trapezoidal rule on the same half contour (fpm(16)=1): the midpoints
 * theta_e = pi (e - 1/2) / ne, e = 1..ne, each with theta-weight pi/ne.  A
 * rule with theta-nodes and weights (theta_e, v_e) gives
 * w_e = (v_e / (i pi)) z'(theta_e) = (v_e r / pi)(a cos theta_e + i sin theta_e),
 * here w_e = (r / ne)(a cos theta_e + i sin theta_e).  With the conjugate
 * lower half these are the 2 ne equally spaced points of the full contour. */
int orc_contour_trapezoid(int ne, double emin, double emax, double ratio, double* z, double* w)
{
    if (ne < 1) return -1;
    double c = 0.5 * (emin + emax), r = 0.5 * (emax - emin);
    for (int e = 0; e < ne; ++e) {
        double th = M_PI * (e + 0.5) / ne;
        z[2 * e] = c + r * cos(th);
        z[2 * e + 1] = ratio * r * sin(th);
        w[2 * e] = r * ratio * cos(th) / ne;
        w[2 * e + 1] = r * sin(th) / ne;
    }
    return 0;
}

/* Jacobi elliptic functions for the Zolotarev rule.  K(m) = pi / (2 AGM(1,
 * sqrt(1-m))); sn and cn by the descending Landen (AGM) scheme: a_0 = 1,
 * b_0 = sqrt(1-m), c_0 = sqrt(m), a_{i+1} = (a_i+b_i)/2, b_{i+1} = sqrt(a_i b_i),
 * c_{i+1} = (a_i-b_i)/2 until c_N is negligible; phi_N = 2^N a_N u and
 * phi_{i-1} = (phi_i + asin(c_i sin(phi_i) / a_i)) / 2; sn = sin phi_0,
 * cn = cos phi_0 (m = k^2 is the parameter). */
double orc_ellipk(double m)
{
    double a = 1.0, b = sqrt(1.0 - m);
    for (int i = 0; i < 60 && fabs(a - b) > 1e-16 * a; ++i) {
        double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
    }
    return M_PI / (2.0 * a);
}

void orc_ellipj(double u, double m, double* sn, double* cn)
{
    double a[64], c[64];
    double b = sqrt(1.0 - m);
    a[0] = 1.0;
    c[0] = sqrt(m);
    int N = 0;
    while (N < 62 && fabs(c[N]) > 1e-16) {
        a[N + 1] = 0.5 * (a[N] + b);
        c[N + 1] = 0.5 * (a[N] - b);
        b = sqrt(a[N] * b);
        ++N;
    }
    double phi = ldexp(a[N] * u, N);
    for (int i = N; i > 0; --i) phi = 0.5 * (phi + asin(c[i] * sin(phi) / a[i]));
    *sn = sin(phi);
    *cn = cos(phi);
}

/* Zolotarev rule (fpm(16)=2).  With x = (lambda - c)/r and the Moebius map
 * u = (1 + x)/(1 - x), the indicator of [Emin, Emax] is (1 + sign(u))/2.
 * Outside a transition band |x -+ 1| < eta at the two edges, u lies in
 * [-R, -1/R] or [1/R, R], R = (2 + eta)/eta; s = u/R lies in
 * [-1, -l] U [l, 1], l = 1/R^2.  Zolotarev's best approximation of sign(s)
 * there among odd rationals of type (2n-1, 2n), n = 2 ne, vanishing at 0 and
 * infinity, is Z(s) = M s prod_{j<ne} (s^2 + c_{2j}) / prod_{j<=ne} (s^2 + c_{2j-1}),
 * c_j = l^2 sn^2(j K'/n; l') / cn^2(j K'/n; l'), l' = sqrt(1 - l^2),
 * K' = K(l'^2), and M = 2 / (max Zhat + min Zhat) over [l, 1] (Zhat = Z/M) so
 * that 1 - Z equioscillates.  The filter rho = (1 + Z(u/R))/2 is a real
 * rational function of lambda with ne conjugate pole pairs; its poles
 * s_k = i sqrt(c_{2k-1}) map to x_k = (R s_k - 1)/(R s_k + 1) on the unit
 * circle, z_k = c + r x_k, and partial fractions give
 * rho(lambda) = rho(inf) + sum_k Re(w_k / (z_k - lambda)),
 * w_k = -nu_k R r (1 - x_k)^2 / 2, nu_k the residue of Z at s_k.  The constant
 * rho(inf) = (1 + Z(-1/R))/2, at most half the approximation error, is
 * dropped (the filter form has no constant term).  Returns 0, or -1 for ne < 1. */
static cplx zolo_hat(int ne, const double* codd, const double* ceven, cplx s)
{
    cplx num = s, den = 1.0;
    for (int j = 0; j < ne - 1; ++j) num *= s * s + ceven[j];
    for (int j = 0; j < ne; ++j) den *= s * s + codd[j];
    return num / den;
}

int orc_contour_zolotarev(int ne, double emin, double emax, double eta, double* z, double* w)
{
    if (ne < 1) return -1;
    const int n = 2 * ne;
    const double R = (2.0 + eta) / eta, l = 1.0 / (R * R), mp = 1.0 - l * l;
    const double Kp = orc_ellipk(mp);
    double* codd = (double*)malloc(sizeof(double) * ne);
    double* ceven = (double*)malloc(sizeof(double) * (ne > 1 ? ne - 1 : 1));
    for (int j = 1; j < n; ++j) {
        double sn, cn;
        orc_ellipj(j * Kp / n, mp, &sn, &cn);
        const double cj = l * l * sn * sn / (cn * cn);
        if (j % 2) codd[j / 2] = cj;
        else ceven[j / 2 - 1] = cj;
    }
    /* extremes of Zhat on [l, 1]: log-spaced grid, then golden-section refinement */
    const int G = 20000;
    double zmin = INFINITY, zmax = -INFINITY;
    for (int g = 0; g <= G; ++g) {
        const double s = l * pow(1.0 / l, (double)g / G);
        const double v = creal(zolo_hat(ne, codd, ceven, s));
        if (v < zmin) zmin = v;
        if (v > zmax) zmax = v;
        if (g > 0 && g < G) {
            const double s0 = l * pow(1.0 / l, (double)(g - 1) / G), s1 = l * pow(1.0 / l, (double)(g + 1) / G);
            const double v0 = creal(zolo_hat(ne, codd, ceven, s0)), v1 = creal(zolo_hat(ne, codd, ceven, s1));
            const int is_max = v >= v0 && v >= v1, is_min = v <= v0 && v <= v1;
            if (is_max || is_min) {
                double a = s0, b = s1;
                const double gr = 0.5 * (sqrt(5.0) - 1.0);
                for (int it = 0; it < 80; ++it) {
                    const double c1 = b - gr * (b - a), c2 = a + gr * (b - a);
                    const double f1 = creal(zolo_hat(ne, codd, ceven, c1)), f2 = creal(zolo_hat(ne, codd, ceven, c2));
                    if (is_max ? f1 > f2 : f1 < f2) b = c2;
                    else a = c1;
                }
                const double ve = creal(zolo_hat(ne, codd, ceven, 0.5 * (a + b)));
                if (ve < zmin) zmin = ve;
                if (ve > zmax) zmax = ve;
            }
        }
    }
    const double M = 2.0 / (zmax + zmin);
    const double c = 0.5 * (emin + emax), r = 0.5 * (emax - emin);
    for (int k = 0; k < ne; ++k) {
        const cplx sk = I * sqrt(codd[k]);
        cplx num = M;
        for (int j = 0; j < ne - 1; ++j) num *= sk * sk + ceven[j];
        double den = 2.0;
        for (int j = 0; j < ne; ++j)
            if (j != k) den *= codd[j] - codd[k];
        const cplx nu = num / den;
        const cplx xk = (R * sk - 1.0) / (R * sk + 1.0);
        const cplx zk = c + r * xk, wk = -nu * R * r * (1.0 - xk) * (1.0 - xk) / 2.0;
        z[2 * k] = creal(zk);
        z[2 * k + 1] = cimag(zk);
        w[2 * k] = creal(wk);
        w[2 * k + 1] = cimag(wk);
    }
    free(codd);
    free(ceven);
    return 0;
}

/* Nodes of the quadrature rule fpm(16): 0 Gauss-Legendre, 1 trapezoidal,
 * 2 Zolotarev (circle, ratio ignored, edge band eta = 0.05). */
static const double kZoloEta = 0.05;

static int contour_nodes(int rule, int ne, double emin, double emax, double ratio, double* z, double* w)
{
    if (rule == 2) return orc_contour_zolotarev(ne, emin, emax, kZoloEta, z, w);
    return rule == 1 ? orc_contour_trapezoid(ne, emin, emax, ratio, z, w)
                     : orc_contour_gauss(ne, emin, emax, ratio, z, w);
}

/* Rational filter rho(lambda) = sum_e Re(w_e / (z_e - lambda)): the scalar the
 * quadrature applies to an eigenvector with eigenvalue lambda. */
double orc_rho(int ne, const double* z, const double* w, double lam)
{
    double s = 0.0;
    for (int e = 0; e < ne; ++e) {
        cplx ze = z[2 * e] + I * z[2 * e + 1];
        cplx we = w[2 * e] + I * w[2 * e + 1];
        s += creal(we / (ze - lam));
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Y = A X for column-major X (n x m). B == NULL means the identity. */
static void csr_mm(const ocsr* A, int m, const double* X, double* Y)
{
    int n = A->n;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < m; ++j) {
        const double* x = X + (size_t)n * j;
        double* y = Y + (size_t)n * j;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int p = A->ip[i]; p < A->ip[i + 1]; ++p) s += A->v[p] * x[A->ix[p]];
            y[i] = s;
        }
    }
}

static void b_mm(const ocsr* B, int n, int m, const double* X, double* Y)
{
    if (B) csr_mm(B, m, X, Y);
    else memcpy(Y, X, sizeof(double) * (size_t)n * m);
}

void orc_csr_mm(int n, const int* ip, const int* ix, const double* v, int m, const double* X, double* Y)
{
    ocsr A = {n, ip, ix, v};
    csr_mm(&A, m, X, Y);
}

/* ------------------------------------------------------------------------ */
/* Banded storage of the lower triangle: L[i*(bw+1) + d] holds element (i, i-d). */
static int csr_bandwidth(const ocsr* A)
{
    int bw = 0;
    for (int i = 0; i < A->n; ++i)
        for (int p = A->ip[i]; p < A->ip[i + 1]; ++p) {
            int d = abs(i - A->ix[p]);
            if (d > bw) bw = d;
        }
    return bw;
}

/* LDL^T of the complex symmetric banded matrix K = zB - A, no pivoting.
 * On return band[i*(bw+1)+0] = d_i and band[i*(bw+1)+k] = l_{i,i-k}. */
static int band_ldlt_complex(int n, int bw, cplx* band)
{
    int ld = bw + 1;
    for (int j = 0; j < n; ++j) {
        /* d_j = K_jj - sum_k l_jk^2 d_k */
        cplx dj = band[(size_t)j * ld];
        int k0 = j - bw < 0 ? 0 : j - bw;
        for (int k = k0; k < j; ++k) {
            cplx ljk = band[(size_t)j * ld + (j - k)];
            dj -= ljk * ljk * band[(size_t)k * ld];
        }
        if (cabs(dj) == 0.0) return -1;
        band[(size_t)j * ld] = dj;
        int i1 = j + bw >= n ? n - 1 : j + bw;
        for (int i = j + 1; i <= i1; ++i) {
            /* l_ij = (K_ij - sum_k l_ik l_jk d_k) / d_j, k < j, k >= i - bw */
            cplx s = band[(size_t)i * ld + (i - j)];
            int kk0 = i - bw > k0 ? i - bw : k0;
            for (int k = kk0; k < j; ++k)
                s -= band[(size_t)i * ld + (i - k)] * band[(size_t)j * ld + (j - k)] * band[(size_t)k * ld];
            band[(size_t)i * ld + (i - j)] = s / dj;
        }
    }
    return 0;
}

static void band_ldlt_solve(int n, int bw, const cplx* band, cplx* x)
{
    int ld = bw + 1;
    for (int i = 0; i < n; ++i) { /* L y = b */
        cplx s = x[i];
        int k0 = i - bw < 0 ? 0 : i - bw;
        for (int k = k0; k < i; ++k) s -= band[(size_t)i * ld + (i - k)] * x[k];
        x[i] = s;
    }
    for (int i = 0; i < n; ++i) x[i] /= band[(size_t)i * ld];
    for (int i = n - 1; i >= 0; --i) { /* L^T x = y */
        cplx s = x[i];
        int k1 = i + bw >= n ? n - 1 : i + bw;
        for (int k = i + 1; k <= k1; ++k) s -= band[(size_t)k * ld + (k - i)] * x[k];
        x[i] = s;
    }
}

static cplx* build_shifted_band(const ocsr* A, const ocsr* B, cplx z, int bw)
{
    int n = A->n, ld = bw + 1;
    cplx* band = (cplx*)calloc((size_t)n * ld, sizeof(cplx));
    if (!band) return NULL;
    for (int i = 0; i < n; ++i)
        for (int p = A->ip[i]; p < A->ip[i + 1]; ++p) {
            int j = A->ix[p];
            if (j <= i) band[(size_t)i * ld + (i - j)] -= A->v[p];
        }
    if (B) {
        for (int i = 0; i < n; ++i)
            for (int p = B->ip[i]; p < B->ip[i + 1]; ++p) {
                int j = B->ix[p];
                if (j <= i) band[(size_t)i * ld + (i - j)] += z * B->v[p];
            }
    } else {
        for (int i = 0; i < n; ++i) band[(size_t)i * ld] += z;
    }
    return band;
}

/* Direct shifted solve: (zB - A) X = RHS for m complex right-hand sides
 * (column-major, interleaved re/im).  Returns 0, or -1 on a zero pivot. */
int orc_shifted_solve_direct(int n, const int* ip, const int* ix, const double* av,
                             const int* bip, const int* bix, const double* bv,
                             double zr, double zi, int m, const double* rhs, double* sol)
{
    ocsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    const ocsr* B = bip ? &Bm : NULL;
    int bw = csr_bandwidth(&A);
    if (B) { int b2 = csr_bandwidth(B); if (b2 > bw) bw = b2; }
    cplx* band = build_shifted_band(&A, B, zr + I * zi, bw);
    if (!band) return -2;
    int st = band_ldlt_complex(n, bw, band);
    if (st == 0) {
        cplx* x = (cplx*)malloc(sizeof(cplx) * n);
        for (int j = 0; j < m; ++j) {
            for (int i = 0; i < n; ++i) x[i] = rhs[2 * ((size_t)n * j + i)] + I * rhs[2 * ((size_t)n * j + i) + 1];
            band_ldlt_solve(n, bw, band, x);
            for (int i = 0; i < n; ++i) {
                sol[2 * ((size_t)n * j + i)] = creal(x[i]);
                sol[2 * ((size_t)n * j + i) + 1] = cimag(x[i]);
            }
        }
        free(x);
    }
    free(band);
    return st;
}

/* ------------------------------------------------------------------------ */
/* FP64 COCG (conjugate orthogonal CG) for one complex symmetric system
 * (zB - A) x = b, x0 = 0; unconjugated inner products u^T v.  Stops when
 * ||r||_2 <= tol ||b||_2 or after maxit steps.  Returns the iteration count,
 * or -1 on breakdown (p^T K p == 0). */
static void shifted_apply(const ocsr* A, const ocsr* B, cplx z, const cplx* p, cplx* q)
{
    int n = A->n;
    for (int i = 0; i < n; ++i) {
        cplx s = 0.0;
        for (int k = A->ip[i]; k < A->ip[i + 1]; ++k) s -= A->v[k] * p[A->ix[k]];
        if (B) {
            cplx t = 0.0;
            for (int k = B->ip[i]; k < B->ip[i + 1]; ++k) t += B->v[k] * p[B->ix[k]];
            s += z * t;
        } else {
            s += z * p[i];
        }
        q[i] = s;
    }
}

static int cocg_one(const ocsr* A, const ocsr* B, cplx z, const cplx* b, cplx* x, double tol, int maxit)
{
    int n = A->n;
    cplx* r = (cplx*)malloc(sizeof(cplx) * n);
    cplx* p = (cplx*)malloc(sizeof(cplx) * n);
    cplx* q = (cplx*)malloc(sizeof(cplx) * n);
    double bn = 0.0;
    cplx rho = 0.0;
    for (int i = 0; i < n; ++i) {
        x[i] = 0.0;
        r[i] = b[i];
        p[i] = b[i];
        bn += creal(b[i]) * creal(b[i]) + cimag(b[i]) * cimag(b[i]);
        rho += b[i] * b[i];
    }
    bn = sqrt(bn);
    int it = 0, status = 0;
    if (bn == 0.0) goto done;
    for (it = 0; it < maxit; ++it) {
        shifted_apply(A, B, z, p, q);
        cplx sig = 0.0;
        for (int i = 0; i < n; ++i) sig += p[i] * q[i];
        if (sig == 0.0) { status = -1; break; }
        cplx alpha = rho / sig;
        double rn = 0.0;
        cplx rho1 = 0.0;
        for (int i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            rn += creal(r[i]) * creal(r[i]) + cimag(r[i]) * cimag(r[i]);
            rho1 += r[i] * r[i];
        }
        if (sqrt(rn) <= tol * bn) { ++it; break; }
        cplx beta = rho1 / rho;
        rho = rho1;
        for (int i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
done:
    free(r); free(p); free(q);
    return status ? status : it;
}

int orc_shifted_solve_cocg(int n, const int* ip, const int* ix, const double* av,
                           const int* bip, const int* bix, const double* bv,
                           double zr, double zi, int m, const double* rhs, double* sol,
                           double tol, int maxit, int* iters)
{
    ocsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    const ocsr* B = bip ? &Bm : NULL;
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
    for (int j = 0; j < m; ++j) {
        cplx* b = (cplx*)malloc(sizeof(cplx) * n);
        cplx* x = (cplx*)malloc(sizeof(cplx) * n);
        for (int i = 0; i < n; ++i) b[i] = rhs[2 * ((size_t)n * j + i)] + I * rhs[2 * ((size_t)n * j + i) + 1];
        int it = cocg_one(&A, B, zr + I * zi, b, x, tol, maxit);
        if (it < 0) bad++;
        if (iters) iters[j] = it;
        for (int i = 0; i < n; ++i) {
            sol[2 * ((size_t)n * j + i)] = creal(x[i]);
            sol[2 * ((size_t)n * j + i) + 1] = cimag(x[i]);
        }
        free(b); free(x);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigensolver for a dense symmetric n x n matrix (column-major,
 * destroyed).  Rotation for the pair (p,q): tau = (a_qq - a_pp)/(2 a_pq),
 * t = sign(tau)/(|tau| + sqrt(1+tau^2)), c = 1/sqrt(1+t^2), s = t c
 * (Golub & Van Loan, symmetric Schur decomposition).  Sweeps until the
 * off-diagonal Frobenius norm is <= 1e-15 of the full norm.  Eigenvalues come
 * out ascending with matching columns of V. */
int orc_jacobi_eig(int n, double* a, double* w, double* V)
{
#define A_(i, j) a[(size_t)(j) * n + (i)]
#define V_(i, j) V[(size_t)(j) * n + (i)]
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) V_(i, j) = (i == j);
    double fro = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) fro += a[k] * a[k];
    fro = sqrt(fro);
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                if (i != j) off += A_(i, j) * A_(i, j);
        if (sqrt(off) <= 1e-15 * fro || fro == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A_(p, q);
                if (apq == 0.0) continue;
                double tau = (A_(q, q) - A_(p, p)) / (2.0 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) { /* A <- A J (columns p, q) */
                    double akp = A_(k, p), akq = A_(k, q);
                    A_(k, p) = c * akp - s * akq;
                    A_(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* A <- J^T A (rows p, q) */
                    double apk = A_(p, k), aqk = A_(q, k);
                    A_(p, k) = c * apk - s * aqk;
                    A_(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V_(k, p), vkq = V_(k, q);
                    V_(k, p) = c * vkp - s * vkq;
                    V_(k, q) = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A_(i, i);
    /* selection sort ascending, permuting V's columns alongside */
    for (int i = 0; i < n; ++i) {
        int k = i;
        for (int j = i + 1; j < n; ++j)
            if (w[j] < w[k]) k = j;
        if (k != i) {
            double t = w[i]; w[i] = w[k]; w[k] = t;
            for (int r = 0; r < n; ++r) { double u = V_(r, i); V_(r, i) = V_(r, k); V_(r, k) = u; }
        }
    }
    return sweep;
#undef A_
#undef V_
}

/* Reduced generalized problem Aq v = lambda Bq v (m x m, column-major,
 * symmetrised on entry).  Route: scale by D = diag(Bq)^{-1/2}; Jacobi on
 * D Bq D = U diag(d) U^T; keep d_i > 1e-14 max d; S = D U_k d_k^{-1/2};
 * Jacobi on S^T Aq S = W Lambda W^T; V = S W (so V^T Bq V = I).  Returns 0 and
 * the kept count in *mk, or -3 when Bq has no positive direction. */
int orc_reduced_gev(int m, const double* Aq, const double* Bq, double* lam, double* V, int* mk)
{
    size_t mm = (size_t)m * m;
    double* dsc = (double*)malloc(sizeof(double) * m);
    double* b = (double*)malloc(sizeof(double) * mm);
    double* a = (double*)malloc(sizeof(double) * mm);
    double* U = (double*)malloc(sizeof(double) * mm);
    double* d = (double*)malloc(sizeof(double) * m);
    int info = 0;
    for (int i = 0; i < m; ++i) {
        double bii = Bq[(size_t)i * m + i];
        dsc[i] = bii > 0.0 ? 1.0 / sqrt(bii) : 0.0;
    }
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
            b[(size_t)j * m + i] = 0.5 * (Bq[(size_t)j * m + i] + Bq[(size_t)i * m + j]) * dsc[i] * dsc[j];
            a[(size_t)j * m + i] = 0.5 * (Aq[(size_t)j * m + i] + Aq[(size_t)i * m + j]) * dsc[i] * dsc[j];
        }
    orc_jacobi_eig(m, b, d, U);
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) if (d[i] > dmax) dmax = d[i];
    int k = 0;
    if (dmax > 0.0)
        for (int i = 0; i < m; ++i) if (d[i] > 1e-14 * dmax) ++k;
    if (k == 0) { info = -3; *mk = 0; goto out; }
    {
        /* S (m x k): column c = D U[:, i_c] / sqrt(d_i), kept in descending d */
        double* S = (double*)malloc(sizeof(double) * (size_t)m * k);
        int c = 0;
        for (int i = m - 1; i >= 0 && c < k; --i) {
            if (!(d[i] > 1e-14 * dmax)) continue;
            double sc = 1.0 / sqrt(d[i]);
            for (int r = 0; r < m; ++r) S[(size_t)c * m + r] = dsc[r] * U[(size_t)i * m + r] * sc;
            ++c;
        }
        /* Aq scaled back: C = S^T Aq S with the symmetrised Aq */
        double* AS = (double*)malloc(sizeof(double) * (size_t)m * k);
        double* C = (double*)malloc(sizeof(double) * (size_t)k * k);
        double* W = (double*)malloc(sizeof(double) * (size_t)k * k);
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < m; ++i) {
                double s = 0.0;
                for (int l = 0; l < m; ++l)
                    s += 0.5 * (Aq[(size_t)l * m + i] + Aq[(size_t)i * m + l]) * S[(size_t)j * m + l];
                AS[(size_t)j * m + i] = s;
            }
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < k; ++i) {
                double s = 0.0;
                for (int l = 0; l < m; ++l) s += S[(size_t)i * m + l] * AS[(size_t)j * m + l];
                C[(size_t)j * k + i] = s;
            }
        for (int j = 0; j < k; ++j) /* symmetrise before Jacobi */
            for (int i = j + 1; i < k; ++i) {
                double s = 0.5 * (C[(size_t)j * k + i] + C[(size_t)i * k + j]);
                C[(size_t)j * k + i] = s;
                C[(size_t)i * k + j] = s;
            }
        orc_jacobi_eig(k, C, lam, W);
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < m; ++i) {
                double s = 0.0;
                for (int l = 0; l < k; ++l) s += S[(size_t)l * m + i] * W[(size_t)j * k + l];
                V[(size_t)j * m + i] = s;
            }
        *mk = k;
        free(S); free(AS); free(C); free(W);
    }
out:
    free(dsc); free(b); free(a); free(U); free(d);
    return info;
}

/* ------------------------------------------------------------------------ */
/* Sylvester inertia: number of negative pivots of A - sigma B from a real
 * banded LDL^T without pivoting (for a tridiagonal matrix this is the Sturm
 * count).  By Sylvester's law of inertia it equals the number of eigenvalues of
 * (A, B) below sigma.  Returns -1 if an exact zero pivot is met. */
long orc_count_below(int n, const int* ip, const int* ix, const double* av,
                     const int* bip, const int* bix, const double* bv, double sigma)
{
    ocsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    const ocsr* B = bip ? &Bm : NULL;
    int bw = csr_bandwidth(&A);
    if (B) { int b2 = csr_bandwidth(B); if (b2 > bw) bw = b2; }
    int ld = bw + 1;
    double* band = (double*)calloc((size_t)n * ld, sizeof(double));
    if (!band) return -2;
    for (int i = 0; i < n; ++i)
        for (int p = ip[i]; p < ip[i + 1]; ++p)
            if (ix[p] <= i) band[(size_t)i * ld + (i - ix[p])] += av[p];
    if (B) {
        for (int i = 0; i < n; ++i)
            for (int p = bip[i]; p < bip[i + 1]; ++p)
                if (bix[p] <= i) band[(size_t)i * ld + (i - bix[p])] -= sigma * bv[p];
    } else {
        for (int i = 0; i < n; ++i) band[(size_t)i * ld] -= sigma;
    }
    long neg = 0;
    for (int j = 0; j < n; ++j) {
        double dj = band[(size_t)j * ld];
        int k0 = j - bw < 0 ? 0 : j - bw;
        for (int k = k0; k < j; ++k) {
            double l = band[(size_t)j * ld + (j - k)];
            dj -= l * l * band[(size_t)k * ld];
        }
        if (dj == 0.0) { free(band); return -1; }
        band[(size_t)j * ld] = dj;
        if (dj < 0) ++neg;
        int i1 = j + bw >= n ? n - 1 : j + bw;
        for (int i = j + 1; i <= i1; ++i) {
            double s = band[(size_t)i * ld + (i - j)];
            int kk0 = i - bw > k0 ? i - bw : k0;
            for (int k = kk0; k < j; ++k)
                s -= band[(size_t)i * ld + (i - k)] * band[(size_t)j * ld + (j - k)] * band[(size_t)k * ld];
            band[(size_t)i * ld + (i - j)] = s / dj;
        }
    }
    free(band);
    return neg;
}

/* ------------------------------------------------------------------------ */
/* Relative residuals res_j = ||A x_j - lambda_j B x_j|| / ||alpha B x_j||,
 * alpha = max(|Emin|, |Emax|) (guide Sec. 3.2, argument res). */
void orc_residuals(int n, const int* ip, const int* ix, const double* av,
                   const int* bip, const int* bix, const double* bv,
                   int m, const double* X, const double* lam, double emin, double emax, double* res)
{
    ocsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    const ocsr* B = bip ? &Bm : NULL;
    double alpha = fmax(fabs(emin), fabs(emax));
    double* AX = (double*)malloc(sizeof(double) * (size_t)n * m);
    double* BX = (double*)malloc(sizeof(double) * (size_t)n * m);
    csr_mm(&A, m, X, AX);
    b_mm(B, n, m, X, BX);
    for (int j = 0; j < m; ++j) {
        double rn = 0.0, bn = 0.0;
        for (int i = 0; i < n; ++i) {
            double r = AX[(size_t)j * n + i] - lam[j] * BX[(size_t)j * n + i];
            rn += r * r;
            bn += BX[(size_t)j * n + i] * BX[(size_t)j * n + i];
        }
        res[j] = sqrt(rn) / (alpha * sqrt(bn));
    }
    free(AX); free(BX);
}

/* ------------------------------------------------------------------------ */
/* Quadrature filter  Q = sum_e Re(w_e (z_e B - A)^{-1} B Y)  (classic form).
 * solver: 0 = banded LDL^T, 1 = COCG to solve_tol.  Returns 0 or -2. */
static int filter_classic(const ocsr* A, const ocsr* B, int ne, const double* z, const double* w,
                          int m, const double* Y, double* Q, int solver, double solve_tol, long* iters)
{
    int n = A->n;
    double* BY = (double*)malloc(sizeof(double) * (size_t)n * m);
    b_mm(B, n, m, Y, BY);
    double* rhs = (double*)malloc(sizeof(double) * 2 * (size_t)n * m);
    for (size_t k = 0; k < (size_t)n * m; ++k) { rhs[2 * k] = BY[k]; rhs[2 * k + 1] = 0.0; }
    double* sol = (double*)malloc(sizeof(double) * 2 * (size_t)n * m);
    int* it = (int*)malloc(sizeof(int) * m);
    memset(Q, 0, sizeof(double) * (size_t)n * m);
    int st = 0;
    for (int e = 0; e < ne && st == 0; ++e) {
        int s;
        if (solver == 0)
            s = orc_shifted_solve_direct(n, A->ip, A->ix, A->v, B ? B->ip : NULL, B ? B->ix : NULL,
                                         B ? B->v : NULL, z[2 * e], z[2 * e + 1], m, rhs, sol);
        else {
            s = orc_shifted_solve_cocg(n, A->ip, A->ix, A->v, B ? B->ip : NULL, B ? B->ix : NULL,
                                       B ? B->v : NULL, z[2 * e], z[2 * e + 1], m, rhs, sol,
                                       solve_tol, 100000, it);
            if (iters) for (int j = 0; j < m; ++j) *iters += it[j] > 0 ? it[j] : 0;
        }
        if (s) { st = -2; break; }
        double wr = w[2 * e], wi = w[2 * e + 1];
        for (size_t k = 0; k < (size_t)n * m; ++k) Q[k] += wr * sol[2 * k] - wi * sol[2 * k + 1];
    }
    free(BY); free(rhs); free(sol); free(it);
    return st;
}

/* Residual-inverse-iteration form of the same filter on the Ritz block X with
 * Ritz values lam:  for every column, (zB-A)^{-1} B x = [x + (zB-A)^{-1}(Ax - lam Bx)]/(z - lam),
 * so Q = X diag(rho(lam)) + sum_e Re(w_e/(z_e - lam_j) Y_e), (z_e B - A) Y_e = A X - B X Lam.
 * Pinned by tests against the dense spectral formula X diag(rho) X^T B applied to
 * the Ritz pairs of a random subspace (not eigenpairs), and against filter_classic. */
static int filter_rii(const ocsr* A, const ocsr* B, int ne, const double* z, const double* w,
                      int m, const double* X, const double* lam, double* Q, int solver,
                      double solve_tol, long* iters)
{
    int n = A->n;
    double* AX = (double*)malloc(sizeof(double) * (size_t)n * m);
    double* BX = (double*)malloc(sizeof(double) * (size_t)n * m);
    csr_mm(A, m, X, AX);
    b_mm(B, n, m, X, BX);
    double* rhs = (double*)malloc(sizeof(double) * 2 * (size_t)n * m);
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < n; ++i) {
            size_t k = (size_t)j * n + i;
            rhs[2 * k] = AX[k] - lam[j] * BX[k];
            rhs[2 * k + 1] = 0.0;
        }
    double* sol = (double*)malloc(sizeof(double) * 2 * (size_t)n * m);
    int* it = (int*)malloc(sizeof(int) * m);
    for (int j = 0; j < m; ++j) {
        double rj = orc_rho(ne, z, w, lam[j]);
        for (int i = 0; i < n; ++i) Q[(size_t)j * n + i] = rj * X[(size_t)j * n + i];
    }
    int st = 0;
    for (int e = 0; e < ne; ++e) {
        int s;
        if (solver == 0)
            s = orc_shifted_solve_direct(n, A->ip, A->ix, A->v, B ? B->ip : NULL, B ? B->ix : NULL,
                                         B ? B->v : NULL, z[2 * e], z[2 * e + 1], m, rhs, sol);
        else {
            s = orc_shifted_solve_cocg(n, A->ip, A->ix, A->v, B ? B->ip : NULL, B ? B->ix : NULL,
                                       B ? B->v : NULL, z[2 * e], z[2 * e + 1], m, rhs, sol,
                                       solve_tol, 100000, it);
            if (iters) for (int j = 0; j < m; ++j) *iters += it[j] > 0 ? it[j] : 0;
        }
        if (s) { st = -2; break; }
        cplx ze = z[2 * e] + I * z[2 * e + 1], we = w[2 * e] + I * w[2 * e + 1];
        for (int j = 0; j < m; ++j) {
            cplx c = we / (ze - lam[j]);
            double cr = creal(c), ci = cimag(c);
            for (int i = 0; i < n; ++i) {
                size_t k = (size_t)j * n + i;
                Q[k] += cr * sol[2 * k] - ci * sol[2 * k + 1];
            }
        }
    }
    free(AX); free(BX); free(rhs); free(sol); free(it);
    return st;
}

/* Exported filter passes on a block (column-major n x m): rii = 0 applies the
 * classic quadrature to Y; rii = 1 the residual-inverse form to (X = Y, lam);
 * rule as fpm(16). */
int orc_filter(int n, const int* ip, const int* ix, const double* av,
               const int* bip, const int* bix, const double* bv,
               int ne, double emin, double emax, double ratio, int m, const double* Y,
               const double* lam, int rii, double* Q, int solver, double solve_tol, int rule)
{
    ocsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    const ocsr* B = bip ? &Bm : NULL;
    double* z = (double*)malloc(sizeof(double) * 2 * ne);
    double* w = (double*)malloc(sizeof(double) * 2 * ne);
    contour_nodes(rule, ne, emin, emax, ratio, z, w);
    int st = rii ? filter_rii(&A, B, ne, z, w, m, Y, lam, Q, solver, solve_tol, NULL)
                 : filter_classic(&A, B, ne, z, w, m, Y, Q, solver, solve_tol, NULL);
    free(z);
    free(w);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Stochastic estimate of the number of eigenvalues inside the contour
 * (fpm(14)=2; the guide cites Di Napoli, Polizzi and Saad for the method).
 * The quadrature filter applied to a vector is rho(B^{-1}A) y, and
 * trace(rho(B^{-1}A)) = sum_i rho(lambda_i), which counts the eigenvalues
 * inside (rho ~ 1) and ignores those far outside (rho ~ 0).  For probes with
 * E[y y^T] = I, E[y^T rho(B^{-1}A) y] is that trace, so the estimate is the
 * mean over the m columns of Y (column-major n x m) of y_j^T Q_j with
 * Q = sum_e Re(w_e (z_e B - A)^{-1} B Y); *sem is the standard error of that
 * mean (sample standard deviation / sqrt(m)).  Returns 0 or -2. */
int orc_stochastic_count(int n, const int* ip, const int* ix, const double* av,
                         const int* bip, const int* bix, const double* bv,
                         int ne, double emin, double emax, double ratio, int m, const double* Y,
                         int solver, double solve_tol, double* est, double* sem, int rule)
{
    double* Q = (double*)malloc(sizeof(double) * (size_t)n * m);
    int st = orc_filter(n, ip, ix, av, bip, bix, bv, ne, emin, emax, ratio, m, Y, NULL, 0, Q, solver, solve_tol,
                        rule);
    if (st) { free(Q); return st; }
    double sum = 0.0, sum2 = 0.0;
    for (int j = 0; j < m; ++j) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += Y[(size_t)j * n + i] * Q[(size_t)j * n + i];
        sum += t;
        sum2 += t * t;
    }
    const double mean = sum / m;
    const double var = m > 1 ? (sum2 - m * mean * mean) / (m - 1) : 0.0;
    *est = mean;
    *sem = sqrt(var > 0.0 ? var : 0.0) / sqrt((double)m);
    free(Q);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FEAST for real symmetric CSR problems (dfeast_scsr{ev,gv} semantics).
 * fpm is the 64-entry parameter array, C indexing fpm[i-1] = fpm(i).
 * Used entries: fpm(2) = Ne, fpm(3) = tolerance exponent, fpm(4) = max
 * refinement loops, fpm(5) = initial subspace given in X, fpm(18) = ellipse ratio.
 * Y0 (n x m0, column-major) is the random start block when fpm(5)=0.
 * On exit: E[0..M-1] inside [Emin,Emax] ascending, E[M..mk-1] outside
 * ascending; X (n x m0) the matching B-orthonormal Ritz vectors; res the
 * relative residuals; *m0 the kept subspace size.  rii selects the RII form of
 * the refinement filter.  Returns info (0, 1, 2, 3, -2, -3, 200, 201, 202). */
int orc_feast_scsr(int n, const int* ip, const int* ix, const double* av,
                   const int* bip, const int* bix, const double* bv,
                   const int* fpm, double emin, double emax, int* m0io,
                   const double* Y0, double* E, double* X, double* res,
                   int* Mout, int* loop_out, double* epsout, int solver, double solve_tol,
                   int rii, double* trace_hist, double* maxres_hist, long* inner_iters)
{
    int m0 = *m0io;
    if (n <= 0) return 202;
    if (m0 <= 0 || m0 > n) return 201;
    if (!(emin < emax)) return 200;
    int ne = fpm[1];
    if (ne < 1) return 102;
    if (fpm[15] < 0 || fpm[15] > 2) return 116;
    ocsr A = {n, ip, ix, av}, Bm = {n, bip, bix, bv};
    const ocsr* B = bip ? &Bm : NULL;
    double ratio = fpm[17] / 100.0;
    double eps = pow(10.0, -fpm[2]);
    int maxloop = fpm[3];
    double alpha = fmax(fabs(emin), fabs(emax));
    double* z = (double*)malloc(sizeof(double) * 2 * ne);
    double* w = (double*)malloc(sizeof(double) * 2 * ne);
    contour_nodes(fpm[15], ne, emin, emax, ratio, z, w);

    size_t nm = (size_t)n * m0;
    double* Q = (double*)malloc(sizeof(double) * nm);
    double* AQ = (double*)malloc(sizeof(double) * nm);
    double* BQ = (double*)malloc(sizeof(double) * nm);
    double* Aq = (double*)malloc(sizeof(double) * m0 * m0);
    double* Bq = (double*)malloc(sizeof(double) * m0 * m0);
    double* V = (double*)malloc(sizeof(double) * m0 * m0);
    double* lam = (double*)malloc(sizeof(double) * m0);
    double* Xw = (double*)calloc(nm, sizeof(double));
    double* rw = (double*)malloc(sizeof(double) * m0);
    int info = 0, k = 0, mk = m0, M = 0;
    double trace_prev = 0.0, eo = 1.0;
    long iters = 0;

    if (fpm[4] == 1) {
        /* initial subspace given: filter it directly (classic form) */
        if (filter_classic(&A, B, ne, z, w, m0, X, Q, solver, solve_tol, &iters)) { info = -2; goto out; }
    } else {
        if (filter_classic(&A, B, ne, z, w, m0, Y0, Q, solver, solve_tol, &iters)) { info = -2; goto out; }
    }
    for (k = 0;; ++k) {
        /* Rayleigh-Ritz: Aq = Q^T A Q, Bq = Q^T B Q */
        csr_mm(&A, mk, Q, AQ);
        b_mm(B, n, mk, Q, BQ);
#pragma omp parallel for schedule(dynamic)
        for (int j = 0; j < mk; ++j)
            for (int i = 0; i < mk; ++i) {
                double sa = 0.0, sb = 0.0;
                for (int r = 0; r < n; ++r) {
                    sa += Q[(size_t)i * n + r] * AQ[(size_t)j * n + r];
                    sb += Q[(size_t)i * n + r] * BQ[(size_t)j * n + r];
                }
                Aq[(size_t)j * mk + i] = sa;
                Bq[(size_t)j * mk + i] = sb;
            }
        int mk2 = 0;
        if (orc_reduced_gev(mk, Aq, Bq, lam, V, &mk2)) { info = -3; goto out; }
        /* X = Q V (n x mk2) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < mk2; ++j)
            for (int r = 0; r < n; ++r) {
                double s = 0.0;
                for (int l = 0; l < mk; ++l) s += Q[(size_t)l * n + r] * V[(size_t)j * mk + l];
                Xw[(size_t)j * n + r] = s;
            }
        mk = mk2;
        orc_residuals(n, ip, ix, av, bip, bix, bv, mk, Xw, lam, emin, emax, rw);
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
        if (trace_hist) trace_hist[k] = trace;
        if (maxres_hist) maxres_hist[k] = M ? maxres : 1.0;
        if (M >= 1 && maxres < eps) { info = 0; break; }
        if (M == 0 && k >= 1) { info = 1; break; }
        if (k >= maxloop) { info = 2; break; }
        int st = rii ? filter_rii(&A, B, ne, z, w, mk, Xw, lam, Q, solver, solve_tol, &iters)
                     : filter_classic(&A, B, ne, z, w, mk, Xw, Q, solver, solve_tol, &iters);
        if (st) { info = -2; goto out; }
    }
    if (info == 0 && M >= mk) info = 3;
    /* order: inside ascending, then outside ascending (lam already ascending) */
    {
        int c = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < mk; ++j) {
                int in = lam[j] >= emin && lam[j] <= emax;
                if ((pass == 0) != in) continue;
                E[c] = lam[j];
                res[c] = rw[j];
                memcpy(X + (size_t)c * n, Xw + (size_t)j * n, sizeof(double) * n);
                ++c;
            }
        for (int j = mk; j < m0; ++j) { E[j] = 0.0; res[j] = 0.0; memset(X + (size_t)j * n, 0, sizeof(double) * n); }
    }
out:
    *Mout = M;
    *loop_out = k;
    *epsout = eo;
    *m0io = mk;
    if (inner_iters) *inner_iters = iters;
    free(z); free(w); free(Q); free(AQ); free(BQ); free(Aq); free(Bq); free(V); free(lam); free(Xw); free(rw);
    return info;
}

/* Gradient of L = sum_k w_k lambda_k with respect to the stored entries of a
 * CSR pattern, for B-orthonormal eigenvectors X (column-major n x m):
 * grad[p] = sum_k w_k X[i_p, k] X[j_p, k] (first-order perturbation of a
 * simple eigenpair; for entries of B pass w_k = -g_k lambda_k). */
void orc_eig_grad(int n, const int* ip, const int* ix, int m, const double* X, const double* w, double* grad)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int p = ip[i]; p < ip[i + 1]; ++p) {
            const int j = ix[p];
            double s = 0.0;
            for (int k = 0; k < m; ++k) s += w[k] * X[(size_t)k * n + i] * X[(size_t)k * n + j];
            grad[p] = s;
        }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
