// Host side of libfeast_gb300: argument checks, contour nodes, the device
// memory plan and the FEAST subspace iteration that drives the kernels.
//
// FEAST v4.0 guide: Sec. 1.1 (algorithm), Sec. 3.1 (fpm and info tables,
// residual inverse iteration and mixed precision tips), Sec. 3.2 (driver
// arguments), Sec. 4.1 (CSR storage), Sec. 4.2 (search contour).
//
// One iteration, all on the device:
//   filter  : COCG over every (node, column) pair, Q accumulated in FP64
//   project : T = A Q, A_Q = Q^T T, B_Q = Q^T (B Q)           (FP64)
//   reduce  : A_Q v = lambda B_Q v by two Jacobi decompositions (FP64)
//   Ritz    : X = Q V, R = A X - B X Lambda, residual norms    (FP64)
// and only the m0 Ritz values and residuals come back to the host, which
// decides convergence.  The first filter pass applies the quadrature to the
// start block (right-hand side B Y); every later pass uses the residual
// inverse form (right-hand side R, see k_filter.cu), which keeps the
// single-precision solves from limiting the FP64 accuracy of the result.
#include <algorithm>
#include <complex>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/feast_gb300.h"
#include "feast_internal.cuh"

using namespace feast;

static thread_local std::string g_err;

extern "C" const char* feast_last_error(void) { return g_err.c_str(); }

namespace feast {
const char* set_last_error(const char* msg)
{
    g_err = msg;
    return g_err.c_str();
}
}  // namespace feast

static int cuda_fail(cudaError_t e, const char* where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return -4;
}

#define CK(x)                                             \
    do {                                                  \
        cudaError_t _e = (x);                             \
        if (_e != cudaSuccess) return cuda_fail(_e, #x);  \
    } while (0)

// ---------------------------------------------------------------- fpm
extern "C" int feast_init(int* fpm)
{
    for (int i = 0; i < 64; ++i) fpm[i] = 0;
    const int def[][2] = {{1, 0},  {2, 8},  {3, 12}, {4, 20},  {5, 0},  {6, 1},  {8, 16},
                          {10, 1}, {14, 0}, {15, 2}, {16, 0},  {18, 30}, {19, 0}, {40, 0},
                          {41, 1}, {42, 1}, {43, 0}, {45, 1},  {46, 40}};
    for (auto& d : def) fpm[d[0] - 1] = d[1];
    return 0;
}

static bool gauss_ne_ok(int ne)
{
    return (ne >= 1 && ne <= 20) || ne == 24 || ne == 32 || ne == 40 || ne == 48 || ne == 56;
}

static constexpr int kMaxTrapezoidNodes = 1024;

static int check_fpm(const int* fpm)
{
    if (fpm[15] < 0 || fpm[15] > 2) return 116;
    if (fpm[15] != 1 ? !gauss_ne_ok(fpm[1]) : (fpm[1] < 1 || fpm[1] > kMaxTrapezoidNodes)) return 102;
    if (fpm[2] < 0 || fpm[2] > 16) return 103;
    if (fpm[3] < 0) return 104;
    if (fpm[4] != 0 && fpm[4] != 1) return 105;
    if (fpm[5] != 0 && fpm[5] != 1) return 106;
    if (fpm[13] < 0 || fpm[13] > 2) return 114;
    if (fpm[17] <= 0) return 118;
    if (fpm[39] < -1 || fpm[39] > 1) return 140;
    if (fpm[41] != 0 && fpm[41] != 1) return 142;
    if (fpm[44] < 0 || fpm[44] > 16) return 145;
    if (fpm[45] < 1) return 146;
    if (fpm[49] < 0) return 150;
    if (fpm[50] < 0) return 151;
    if (fpm[53] != 0 && fpm[53] != 1) return 154;
    return 0;
}

// ---------------------------------------------------------------- contour
// Gauss-Legendre rule by Newton's method on P_n, started from Tricomi's
// asymptotic roots; P_n and P_n' from the three-term recurrence.
static void gl_rule(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int k = 1; k <= n; ++k) {
        const double th = M_PI * (4.0 * k - 1.0) / (4.0 * n + 2.0);
        double t = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(th);
        double d = 0.0;
        for (int it = 0; it < 60; ++it) {
            double pm = 1.0, p = t;  // P_0, P_1
            for (int j = 2; j <= n; ++j) {
                const double pn = ((2.0 * j - 1.0) * t * p - (j - 1.0) * pm) / j;
                pm = p;
                p = pn;
            }
            if (n == 1) { p = t; pm = 1.0; }
            d = n * (pm - t * p) / (1.0 - t * t);
            const double step = p / d;
            t -= step;
            if (std::fabs(step) <= 1e-17 * (1.0 + std::fabs(t))) break;
        }
        double pm = 1.0, p = t;
        for (int j = 2; j <= n; ++j) {
            const double pn = ((2.0 * j - 1.0) * t * p - (j - 1.0) * pm) / j;
            pm = p;
            p = pn;
        }
        if (n == 1) { p = t; pm = 1.0; }
        d = n * (pm - t * p) / (1.0 - t * t);
        x[k - 1] = t;
        w[k - 1] = 2.0 / ((1.0 - t * t) * d * d);
    }
}

// zw[4e..4e+3] = (Re z_e, Im z_e, Re w_e, Im w_e)
// ---------------------------------------------------------------- Zolotarev rule
// Complete elliptic integral K(m) by the arithmetic-geometric mean, and
// sn(u|m), cn(u|m) by the descending Landen transformation (m = k^2).
static double ell_k(double m)
{
    double a = 1.0, g = std::sqrt(1.0 - m);
    for (int it = 0; it < 64 && std::fabs(a - g) > 4e-16 * a; ++it) {
        const double t = 0.5 * (a + g);
        g = std::sqrt(a * g);
        a = t;
    }
    return M_PI / (2.0 * a);
}

static void ell_sncn(double u, double m, double& sn, double& cn)
{
    std::vector<double> as{1.0}, cs{std::sqrt(m)};
    double b = std::sqrt(1.0 - m);
    while (std::fabs(cs.back()) > 1e-16 && as.size() < 64) {
        const double a = as.back();
        as.push_back(0.5 * (a + b));
        cs.push_back(0.5 * (a - b));
        b = std::sqrt(a * b);
    }
    const int N = (int)as.size() - 1;
    double phi = std::ldexp(as[N] * u, N);
    for (int i = N; i >= 1; --i) phi = 0.5 * (phi + std::asin(cs[i] * std::sin(phi) / as[i]));
    sn = std::sin(phi);
    cn = std::cos(phi);
}

static constexpr double kZolotarevEta = 0.05;  // edge band half-width / interval half-width

// Zolotarev rule (fpm(16) = 2; the guide cites Guettel, Polizzi, Tang and
// Viaud and prints no formula).  With x = (lambda - c)/r and u = (1+x)/(1-x)
// the interval's indicator is (1 + sign u)/2; away from the edge bands
// (|x| <= 1/(1+eta) inside, |x| >= 1+eta outside) s = u/R, R = (2+eta)/eta,
// lies in [-1, -l] U [l, 1], l = 1/R^2.  Zolotarev's best odd rational
// approximation of sign(s) there of type (2n-1, 2n), n = 2 ne:
// Z(s) = M s prod_{j=1}^{ne-1} (s^2 + c_{2j}) / prod_{j=1}^{ne} (s^2 + c_{2j-1}),
// c_j = l^2 sn^2(j K'/n | 1-l^2) / cn^2(j K'/n | 1-l^2), K' = K(1-l^2), with
// M = 2/(max + min of Z/M over [l, 1]).  rho = (1 + Z(u/R))/2 has ne
// conjugate pole pairs on the circle through Emin and Emax: the node of
// s_k = i sqrt(c_{2k-1}) is z_k = c + r x_k, x_k = (R s_k - 1)/(R s_k + 1),
// with weight w_k = -nu_k R r (1 - x_k)^2 / 2 (nu_k: residue of Z at s_k), so
// that rho(lambda) = rho(inf) + sum_k Re(w_k/(z_k - lambda)); the constant
// rho(inf), below half the approximation error, is left out.
static void zolotarev(int ne, double emin, double emax, std::vector<double>& zw)
{
    const int n = 2 * ne;
    const double R = (2.0 + kZolotarevEta) / kZolotarevEta, l = 1.0 / (R * R), mc = 1.0 - l * l;
    const double Kc = ell_k(mc);
    std::vector<double> co(ne), ce(std::max(ne - 1, 0));  // c_{2k-1}, c_{2k}
    for (int j = 1; j < n; ++j) {
        double sn = 0.0, cn = 0.0;
        ell_sncn(j * Kc / n, mc, sn, cn);
        const double cj = l * l * (sn / cn) * (sn / cn);
        if (j & 1) co[(j - 1) / 2] = cj;
        else ce[j / 2 - 1] = cj;
    }
    auto zhat = [&](double sv) {  // Z/M on the positive real axis
        double v = sv;
        for (double c : ce) v *= sv * sv + c;
        for (double c : co) v /= sv * sv + c;
        return v;
    };
    // extremes over [l, 1]: log grid; at each local extremum the vertex of the
    // parabola through its three grid points (error in the value ~ h^4)
    const int G = 40000;
    std::vector<double> t(G + 1), v(G + 1);
    for (int g = 0; g <= G; ++g) {
        t[g] = std::log(l) * (1.0 - (double)g / G);
        v[g] = zhat(std::exp(t[g]));
    }
    double vmin = std::min(v[0], v[G]), vmax = std::max(v[0], v[G]);
    for (int g = 1; g < G; ++g) {
        if ((v[g] - v[g - 1]) * (v[g + 1] - v[g]) > 0.0) continue;
        const double h = t[g + 1] - t[g], curv = v[g + 1] - 2.0 * v[g] + v[g - 1];
        double f = v[g];
        if (curv != 0.0) {
            const double d = std::max(-1.0, std::min(1.0, 0.5 * (v[g - 1] - v[g + 1]) / curv));
            f = zhat(std::exp(t[g] + d * h));
        }
        vmin = std::min(vmin, f);
        vmax = std::max(vmax, f);
    }
    const double M = 2.0 / (vmax + vmin);
    const double c = 0.5 * (emin + emax), r = 0.5 * (emax - emin);
    zw.assign(4 * (size_t)ne, 0.0);
    for (int k = 0; k < ne; ++k) {
        const std::complex<double> sk(0.0, std::sqrt(co[k]));
        std::complex<double> num(M, 0.0);
        for (double cv : ce) num *= sk * sk + cv;
        double den = 2.0;
        for (int j = 0; j < ne; ++j)
            if (j != k) den *= co[j] - co[k];
        const std::complex<double> nu = num / den;
        const std::complex<double> xk = (R * sk - 1.0) / (R * sk + 1.0);
        const std::complex<double> zk = c + r * xk, wk = -nu * (R * r / 2.0) * (1.0 - xk) * (1.0 - xk);
        zw[4 * k] = zk.real();
        zw[4 * k + 1] = zk.imag();
        zw[4 * k + 2] = wk.real();
        zw[4 * k + 3] = wk.imag();
    }
}

// Nodes and weights of the quadrature rule fpm(16) on the upper half of the
// ellipse z(t) = c + r cos t + i a r sin t, t in [0, pi]: a rule with nodes
// t_e and t-weights v_e gives w_e = (v_e / (i pi)) z'(t_e)
// = (v_e r / pi)(a cos t_e + i sin t_e).  rule 0: Gauss-Legendre mapped by
// t = (pi/2)(1 - x), v_e = (pi/2) omega_e; rule 1: trapezoidal (midpoints)
// t_e = pi (e + 1/2) / ne, v_e = pi / ne, which with the conjugate lower
// half are 2 ne equally spaced points of the whole contour.
static void contour(int rule, int ne, double emin, double emax, double ratio, std::vector<double>& zw)
{
    if (rule == 2) {  // Zolotarev: its own nodes on the circle (ratio not used)
        zolotarev(ne, emin, emax, zw);
        return;
    }
    std::vector<double> t(ne), v(ne);
    if (rule == 1) {
        for (int e = 0; e < ne; ++e) {
            t[e] = M_PI * (e + 0.5) / ne;
            v[e] = M_PI / ne;
        }
    } else {
        std::vector<double> x, om;
        gl_rule(ne, x, om);
        for (int e = 0; e < ne; ++e) {
            t[e] = 0.5 * M_PI * (1.0 - x[e]);
            v[e] = 0.5 * M_PI * om[e];
        }
    }
    const double c = 0.5 * (emin + emax), r = 0.5 * (emax - emin);
    zw.assign(4 * (size_t)ne, 0.0);
    for (int e = 0; e < ne; ++e) {
        const double ct = std::cos(t[e]), st = std::sin(t[e]);
        zw[4 * e] = c + r * ct;
        zw[4 * e + 1] = ratio * r * st;
        zw[4 * e + 2] = v[e] / M_PI * r * ratio * ct;
        zw[4 * e + 3] = v[e] / M_PI * r * st;
    }
}

extern "C" int feast_contour_nodes(int ne, double emin, double emax, int ratio_pct, double* z, double* w)
{
    if (!gauss_ne_ok(ne)) return 102;
    if (!(emin < emax)) return 200;
    std::vector<double> zw;
    contour(0, ne, emin, emax, ratio_pct / 100.0, zw);
    for (int e = 0; e < ne; ++e) {
        z[2 * e] = zw[4 * e];
        z[2 * e + 1] = zw[4 * e + 1];
        w[2 * e] = zw[4 * e + 2];
        w[2 * e + 1] = zw[4 * e + 3];
    }
    return 0;
}

extern "C" int feast_contour_nodes_rule(int rule, int ne, double emin, double emax, int ratio_pct, double* z,
                                        double* w)
{
    if (rule < 0 || rule > 2) return 116;
    if (rule != 1 ? !gauss_ne_ok(ne) : (ne < 1 || ne > kMaxTrapezoidNodes)) return 102;
    if (!(emin < emax)) return 200;
    std::vector<double> zw;
    contour(rule, ne, emin, emax, ratio_pct / 100.0, zw);
    for (int e = 0; e < ne; ++e) {
        z[2 * e] = zw[4 * e];
        z[2 * e + 1] = zw[4 * e + 1];
        w[2 * e] = zw[4 * e + 2];
        w[2 * e + 1] = zw[4 * e + 3];
    }
    return 0;
}

extern "C" int feast_filter_layout(int nb, int fp64, int* W, int* nbp, int* mt)
{
    int p = 1;
    while (p < nb) p <<= 1;
    if (p > 32 || nb < 1) return -101;
    const int w = fp64 ? std::max(16, p) : std::max(32, p);
    *W = w;
    *nbp = p;
    *mt = w / p;
    return 0;
}

// ---------------------------------------------------------------- memory plan
namespace {

struct Plan {
    int n = 0, m0 = 0, ne = 0, nbp = 0, nbatch = 0, W = 0, mt = 0, G = 0, RB = 0, nrb = 0;
    int RBb = 0, nrb_b = 0;
    long long nitems = 0, nitems_b = 0;
    bool fp64 = false, hasB = false;
    int nnzA = 0, nnzB = 0;
    int ksplit = 1;
    bool oz = true;  // projections from exact BF16 slice products (fpm(54) = 0) or FP64 DMMA (1)
    bool win = false;  // try the staged-window step A (rows per item automatic, fpm(51) = 0)
    int nslot = 1;  // partial-sum slots per group (item slots + bucket slots)
    int nbk = 1;    // bucket counters per group
    size_t gpart = 0, rpart = 0;
};

struct Bufs {
    void *r = nullptr, *p0 = nullptr, *p1 = nullptr;
    ColState* cs = nullptr;
    double* part = nullptr;
    unsigned* grp_count = nullptr;
    unsigned* bk_count = nullptr;
    int* grp_done = nullptr;
    int* iter_max = nullptr;  // [nbatch]
    int* groups_left = nullptr;
    unsigned long long* work = nullptr;
    FiltProb* probs = nullptr;
    void *apk = nullptr, *bpk = nullptr;  // packed (column, value) CSR entries, rows padded to chunks
    int *app = nullptr, *bpp = nullptr;   // padded row pointers
    void* bd = nullptr;                   // diagonal of B (filter precision) when B is diagonal
    int bmode = 0;
    // step A work items chosen at setup: RB rows per item (plan's RB, or the
    // staged-window variant's wrb rows when wrb > 0)
    int RB = 0, nrb = 0;
    long long nitems = 0;
    int wrb = 0, wgrid = 0, wcapr = 0;
    size_t wsmem = 0;
    int4* whdr = nullptr;  // staged-window tables (k_filter.cu win_build)
    int2* wwin = nullptr;
    void* wpk = nullptr;
    int wcape = 0;
    bool wws = false;  // staged step A in its warp-specialized form (cocg_step_ws)
    int* wstat = nullptr;
    void* dQ = nullptr;                   // per-pass quadrature accumulator (filter precision)
    double* zw = nullptr;
    double *Y = nullptr, *Q = nullptr, *X = nullptr, *T = nullptr, *T2 = nullptr;
    double *Aq = nullptr, *Bq = nullptr, *Vr = nullptr, *lam = nullptr, *res = nullptr;
    double *gpart = nullptr, *rpart = nullptr;
    int* mk = nullptr;
    int* perm = nullptr;
    int* ozex = nullptr;  // column exponents of the sliced projections
    void* ozw = nullptr;  // exponents and slices of the sliced Ritz-vector product
    void* eig = nullptr;
};

size_t cplx_bytes(const Plan& P) { return P.fp64 ? 16 : 8; }

Plan make_plan(int n, int nnzA, int nnzB, int m0, const int* fpm, bool filter_only = false)
{
    Plan P;
    P.n = n;
    P.m0 = m0;
    P.ne = fpm[1];
    P.fp64 = fpm[41] == 0;
    P.hasB = nnzB > 0;
    P.nnzA = nnzA;
    P.nnzB = nnzB;
    int nb = fpm[49] > 0 ? std::min(fpm[49], P.ne) : std::min(P.ne, 16);
    for (;;) {
        feast_filter_layout(nb, P.fp64 ? 1 : 0, &P.W, &P.nbp, &P.mt);
        P.G = (m0 + P.mt - 1) / P.mt;
        const double bytes = 3.0 * P.G * (double)n * P.W * cplx_bytes(P);
        if (fpm[49] > 0 || nb <= 1 || bytes <= 128e9) break;
        nb = (nb + 1) / 2;
    }
    P.nbatch = (P.ne + P.nbp - 1) / P.nbp;
    P.RB = fpm[50] > 0 ? std::min(fpm[50], 512) : 256;
    P.nrb = (n + P.RB - 1) / P.RB;
    P.nitems = (long long)P.G * P.nrb;
    P.RBb = 512;
    P.nrb_b = (n + P.RBb - 1) / P.RBb;
    P.nitems_b = (long long)P.G * P.nrb_b;
    // the staged-window step A publishes one slot per CTA (at most 4 per SM)
    P.win = fpm[50] == 0;
    const int wslots = P.win ? num_sms() * 4 : 0;
    P.nslot = std::max({part_slots(P.nrb), part_slots(P.nrb_b), part_slots(wslots)});
    P.nbk = std::max({part_buckets(P.nrb), part_buckets(P.nrb_b), part_buckets(wslots)});
    if (!filter_only) {
        P.oz = fpm[53] == 0;
        P.gpart = P.oz ? gram_oz_partial_doubles(n, m0, nullptr, nullptr, num_sms())
                       : gram_partial_doubles(n, m0, &P.ksplit, num_sms());
        P.rpart = residual_partial_doubles(n, m0);
    }
    return P;
}

struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <typename T>
    T* take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

size_t carve(const Plan& P, void* base, Bufs& B, bool filter_only = false)
{
    Carver c(base);
    const size_t vec = (size_t)P.G * P.n * P.W * cplx_bytes(P);
    B.r = c.take<char>(vec);
    B.p0 = c.take<char>(vec);
    B.p1 = c.take<char>(vec);
    B.cs = c.take<ColState>((size_t)P.G * P.W);
    B.part = c.take<double>((size_t)P.G * P.nslot * P.W * 4);
    B.grp_count = c.take<unsigned>(P.G);
    B.bk_count = c.take<unsigned>((size_t)P.G * P.nbk);
    B.grp_done = c.take<int>(P.G);
    B.iter_max = c.take<int>(P.nbatch);
    B.groups_left = c.take<int>(2);  // [0] groups still iterating, [1] staged-row wait error
    B.work = c.take<unsigned long long>(1);
    B.probs = c.take<FiltProb>(1);
    const size_t pk = P.fp64 ? 16 : 8;
    B.app = c.take<int>((size_t)P.n + 1);
    B.apk = c.take<char>(((size_t)P.nnzA + 7 * (size_t)P.n) * pk);
    if (P.hasB) {
        B.bpp = c.take<int>((size_t)P.n + 1);
        B.bpk = c.take<char>(((size_t)P.nnzB + 7 * (size_t)P.n) * pk);
        B.bd = c.take<double>((size_t)P.n);
    }
    if (P.win) {
        const size_t nrb32 = ((size_t)P.n + 31) / 32;
        // per row block its local row pointers ((rows + 4) ints: at most 36 per 32 rows
        // for 32- to 80-row blocks, plus one block) and its packed entries
        B.wpk = c.take<char>(((size_t)P.nnzA + 7 * (size_t)P.n) * pk + (nrb32 * 36 + 84) * 4);
        B.whdr = c.take<int4>(nrb32);
        B.wwin = c.take<int2>(nrb32 * kWinMax);
        B.wstat = c.take<int>(4);
    }
    B.dQ = c.take<char>((size_t)P.G * P.mt * P.n * (P.fp64 ? 8 : 4));
    B.zw = c.take<double>(4 * (size_t)P.ne);
    if (filter_only) return c.off + 256;
    const size_t blk = (size_t)P.n * P.m0;
    B.Y = c.take<double>(blk);
    B.Q = c.take<double>(blk);
    B.X = c.take<double>(blk);
    B.T = c.take<double>(blk);
    if (P.hasB) B.T2 = c.take<double>(blk);
    const size_t mm = (size_t)P.m0 * P.m0;
    B.Aq = c.take<double>(mm);
    B.Bq = c.take<double>(mm);
    B.Vr = c.take<double>(mm);
    B.lam = c.take<double>(P.m0);
    B.res = c.take<double>(P.m0);
    B.gpart = c.take<double>(P.gpart);
    B.rpart = c.take<double>(P.rpart);
    B.mk = c.take<int>(1);
    B.perm = c.take<int>(P.m0);
    B.ozex = (int*)c.take<char>(gram_oz_work_bytes(P.m0));
    B.ozw = c.take<char>(P.oz ? gemm_oz_work_bytes(P.n, P.m0, P.m0) : 0);
    B.eig = c.take<char>(reduced_work_bytes(P.m0));
    return c.off + 256;
}

// ---------------------------------------------------------------- small kernels
__global__ void k_col_to_row(int n, int m, const double* xc, double* xr)
{
    const long long total = (long long)n * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / m), j = (int)(idx % m);
        xr[idx] = xc[(size_t)j * n + i];
    }
}

// out column c (column-major) = X row-major column perm[c] for c < mk, else 0
__global__ void k_gather_cols(int n, int m, int mk, const double* xr, const int* perm, double* xc)
{
    const long long total = (long long)n * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx / n), i = (int)(idx % n);
        xc[idx] = c < mk ? xr[(size_t)i * m + perm[c]] : 0.0;
    }
}

// Random start block: standard normal values from a counter-based hash
// (splitmix64 of seed and element index) and the Box-Muller transform.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_random_block(long long total, unsigned long long seed, double* y)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const unsigned long long h1 = splitmix64(seed * 0x100000001B3ull + 2 * (unsigned long long)idx);
        const unsigned long long h2 = splitmix64(seed * 0x100000001B3ull + 2 * (unsigned long long)idx + 1);
        const double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
        y[idx] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

// ---------------------------------------------------------------- extreme-eigenvalue search kernels
// Diagonal of a CSR matrix; *offdiag is set when a row stores a nonzero
// off-diagonal value.
__global__ void k_csr_diag(int n, const int* ia, const int* ja, const double* v, double* d, int* offdiag)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double di = 0.0;
        bool off = false;
        for (int p = ia[i]; p < ia[i + 1]; ++p) {
            if (ja[p] == i) di += v[p];
            else if (v[p] != 0.0) off = true;
        }
        d[i] = di;
        if (off) *offdiag = 1;
    }
}

// Gershgorin discs of the rows: centre m_ii, radius sum_{j != i} |m_ij|, of
// M itself (scale == NULL) or of S^{-1/2} M S^{-1/2} with S = diag(scale).
// Per block: part[2 b] = min(centre - radius), part[2 b + 1] = max(centre + radius).
__global__ void __launch_bounds__(256) k_gersh(int n, const int* ia, const int* ja, const double* v,
                                               const double* scale, double* part)
{
    __shared__ double slo[256], shi[256];
    double lo = INFINITY, hi = -INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double si = scale ? scale[i] : 1.0;
        double c = 0.0, r = 0.0;
        for (int p = ia[i]; p < ia[i + 1]; ++p) {
            const int j = ja[p];
            if (j == i) c += v[p];
            else r += scale ? fabs(v[p]) / sqrt(si * scale[j]) : fabs(v[p]);
        }
        if (scale) c /= si;
        lo = fmin(lo, c - r);
        hi = fmax(hi, c + r);
    }
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + o]);
            shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = slo[0];
        part[2 * blockIdx.x + 1] = shi[0];
    }
}

__global__ void k_negate(long long total, const double* a, double* b)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = -a[i];
}

// Reverse the order of the columns c0 .. c1-1 of a column-major n-row block.
__global__ void k_reverse_cols(int n, int c0, int c1, double* x)
{
    const long long half = (c1 - c0) / 2;
    const long long total = half * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = c0 + (int)(idx / n), i = (int)(idx % n);
        const int o = c1 - 1 - (c - c0);
        const double t = x[(size_t)c * n + i];
        x[(size_t)c * n + i] = x[(size_t)o * n + i];
        x[(size_t)o * n + i] = t;
    }
}

// Optional per-kernel timing (fpm(53) = 1): CUDA events recorded on the
// solve's stream around every COCG launch and every Rayleigh-Ritz phase.
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<size_t, size_t>> a, b;  // cocg_step_a / cocg_step_b launches
    std::vector<std::pair<int, std::pair<size_t, size_t>>> phase;
    double out[20] = {0};
    cudaEvent_t ev()
    {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    size_t mark(cudaStream_t s)
    {
        cudaEvent_t e = ev();
        cudaEventRecord(e, s);
        return used - 1;
    }
    void reset(bool enable)
    {
        on = enable;
        used = 0;
        a.clear();
        b.clear();
        phase.clear();
        for (double& v : out) v = 0.0;
    }
    double ms(size_t i, size_t j)
    {
        float t = 0.f;
        cudaEventElapsedTime(&t, pool[i], pool[j]);
        return t;
    }
};
thread_local Prof g_prof;

int grid_for(long long total)
{
    long long b = (total + 255) / 256;
    const long long cap = (long long)num_sms() * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

struct Csr {
    int n = 0, nnz = 0;
    const int* ia = nullptr;
    const int* ja = nullptr;
    const double* v = nullptr;
};

// One filter pass (all node batches) into B.Q.  rii selects the right-hand
// side R (device row-major n x m0 in B.Y) and the coefficients.
int filter_pass(const Plan& P, Bufs& B, int rii, const double* R, const double* X, int maxit, double tol,
                cudaStream_t s)
{
    FilterArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.probs = B.probs;
    fa.nprob = 1;
    fa.nitems = B.nitems;
    fa.nitems_b = P.nitems_b;
    fa.RBb = P.RBb;
    fa.W = P.W;
    fa.nbp = P.nbp;
    fa.mt = P.mt;
    fa.RB = B.RB;
    fa.hasB = P.hasB ? 1 : 0;
    fa.bmode = B.bmode;
    fa.r = B.r;
    fa.p0 = B.p0;
    fa.p1 = B.p1;
    fa.cs = B.cs;
    fa.part = B.part;
    fa.grp_count = B.grp_count;
    fa.bk_count = B.bk_count;
    fa.nbk = P.nbk;
    fa.grp_done = B.grp_done;
    fa.Q = B.Q;
    fa.dQ = B.dQ;
    fa.tol2 = tol * tol;
    fa.groups_left = B.groups_left;
    fa.work = B.work;
    fa.whdr = B.whdr;
    fa.wwin = B.wwin;
    fa.wpk = B.wpk;
    fa.wcapr = B.wcapr;
    fa.wcape = B.wcape;
    fa.werr = B.groups_left + 1;
    fa.wlimit = wait_limit_cycles();
    int grid_a = 1, grid_b = 1;
    filter_grids(P.fp64, P.W, &grid_a, &grid_b);
    grid_a = B.wrb ? B.wgrid : (int)std::min<long long>(grid_a, B.nitems);
    grid_b = (int)std::min<long long>(grid_b, P.nitems_b);
    const int grid = std::max(grid_a, grid_b);  // filter_init
    fa.nslot = P.nslot;
    CK(cudaMemsetAsync(B.iter_max, 0, sizeof(int) * P.nbatch, s));
    CK(cudaMemsetAsync(B.groups_left + 1, 0, sizeof(int), s));
    auto step_a = [&](int k) -> cudaError_t {
        if (B.wws) return launch_cocg_step_ws(fa, B.wrb, k, grid_a, B.wsmem, s);
        return B.wrb ? launch_cocg_step_aw(fa, P.fp64, B.wrb, k, grid_a, B.wsmem, s)
                     : launch_cocg_step_a(fa, P.fp64, k, grid_a, s);
    };
    // a CTA of the staged-window step A that gave up waiting for its copies
    auto wait_failed = [&](int werr) -> int {
        g_err = "COCG step A: staged-row copies did not complete within the wait limit";
        return werr ? -4 : 0;
    };
    int left = P.G;
    for (int b = 0; b < P.nbatch; ++b) {
        fa.iter_max = B.iter_max + b;
        CK(cudaMemsetAsync(B.grp_count, 0, sizeof(unsigned) * P.G, s));
        CK(cudaMemsetAsync(B.bk_count, 0, sizeof(unsigned) * (size_t)P.G * P.nbk, s));
        CK(cudaMemsetAsync(B.grp_done, 0, sizeof(int) * P.G, s));
        CK(cudaMemcpyAsync(B.groups_left, &left, sizeof(int), cudaMemcpyHostToDevice, s));
        CK(launch_colstate_init(fa, b * P.nbp, rii, s));
        CK(launch_filter_init(fa, P.fp64, R, X, rii, b == 0, grid, s));
        for (int k = 0; k < maxit; ++k) {
            if (g_prof.on) {
                const size_t e0 = g_prof.mark(s);
                CK(step_a(k));
                const size_t e1 = g_prof.mark(s);
                CK(launch_cocg_step_b(fa, P.fp64, k, grid_b, s));
                const size_t e2 = g_prof.mark(s);
                g_prof.a.push_back({e0, e1});
                g_prof.b.push_back({e1, e2});
            } else {
                CK(step_a(k));
                CK(launch_cocg_step_b(fa, P.fp64, k, grid_b, s));
            }
            // every few steps: stop launching once no group iterates any more
            if ((k & 7) == 7 && k + 1 < maxit) {
                int h[2] = {1, 0};
                CK(cudaMemcpyAsync(h, B.groups_left, sizeof(h), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                if (h[1]) return wait_failed(h[1]);
                if (h[0] <= 0) break;
            }
        }
    }
    CK(launch_fold_dq(fa, (long long)P.n * P.m0, P.fp64, s));
    if (B.wrb) {
        int werr = 0;
        CK(cudaMemcpyAsync(&werr, B.groups_left + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (werr) return wait_failed(werr);
    }
    return 0;
}

// Pack a device CSR for the filter kernels: rows padded to chunks of 8
// entries (padded row pointers computed on the host from a copy of ia), or,
// when allow_diag and the matrix is diagonal, just its diagonal values.
// *mode: 1 diagonal, 2 packed.
int pack_matrix(const Csr& M, bool fp64, bool allow_diag, int* d_pp, void* d_pk, void* d_bd, int* mode, cudaStream_t s)
{
    const int n = M.n;
    std::vector<int> ia(n + 1);
    CK(cudaMemcpyAsync(ia.data(), M.ia, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (allow_diag && M.nnz == n && ia[n] - ia[0] == n) {
        std::vector<int> ja(n);
        CK(cudaMemcpyAsync(ja.data(), M.ja, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool diag = true;
        for (int i = 0; i < n && diag; ++i) diag = (ia[i + 1] - ia[i] == 1) && ja[ia[i] - ia[0]] == i;
        if (diag) {
            CK(launch_cast_diag(n, M.ia, M.v, fp64, d_bd, s));
            *mode = 1;
            return 0;
        }
    }
    std::vector<int> pp(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const int len = ia[i + 1] - ia[i];
        pp[i + 1] = pp[i] + (len + 7) / 8 * 8;
    }
    CK(cudaMemcpyAsync(d_pp, pp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
    CK(launch_pack_csr(n, M.ia, M.ja, M.v, d_pp, fp64, d_pk, s));
    CK(cudaStreamSynchronize(s));  // pp is a host temporary
    *mode = 2;
    return 0;
}

// Work items of step A: the staged-window variant with 64, else 32 rows per
// item when the matrix's row blocks fit (windows, shared memory, two CTAs per
// SM) and B is the identity or diagonal; otherwise the plan's rows per item
// with the gather through the caches.
int choose_step_a(const Plan& P, Bufs& B, cudaStream_t s)
{
    B.RB = P.RB;
    B.nrb = P.nrb;
    B.nitems = P.nitems;
    B.wrb = 0;
    B.wws = false;
    if (!P.win || B.bmode == 2) return 0;
#ifndef FEAST_STEP_A_WS
#define FEAST_STEP_A_WS 1  // 0: never the warp-specialized form
#endif
    // warp-specialized form (one CTA per SM, the next item's rows staged while the
    // current one computes), 48 then 32 rows per item, for matrices whose row blocks
    // stage many rows per row; with few (a 7-point stencil stages 5 rows per row),
    // two CTAs per SM each issuing their own copies are faster.  Measured on GB300:
    // 7-point 64^3 4,240 (two CTAs) vs 3,830 GB/s; 27-point 96^3 (9.6 staged rows
    // per row) 2,158 vs 2,362 GB/s.
    constexpr double kWsMinStagedPerRow = 7.0;
    for (const int rbw : {48, 32}) {
        if (!FEAST_STEP_A_WS || P.fp64 || P.W != 32) break;
        int st4[4] = {0, 0, 0, 0};
        CK(cudaMemsetAsync(B.wstat, 0, sizeof(st4), s));
        CK(launch_win_build(P.n, rbw, B.app, B.apk, P.fp64, B.wpk, B.whdr, B.wwin, B.wstat, s));
        CK(cudaMemcpyAsync(st4, B.wstat, sizeof(st4), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (st4[3]) return 0;  // column indices outside [0, n): leave the matrix to the general path
        if (st4[2]) continue;
        const int nrbw = (P.n + rbw - 1) / rbw;
        if ((long long)P.G * nrbw >= (1ll << 31)) continue;
        if ((double)st4[0] < kWsMinStagedPerRow * rbw) break;
        const size_t smem = ws_smem_bytes(P.W, rbw, st4[0], st4[1]);
        if (ws_occupancy(P.fp64, P.W, B.bmode, rbw, P.G, smem) < 1) continue;
        B.wws = true;
        B.wsmem = smem;
        B.wgrid = std::min(num_sms(), nrbw);
        B.wrb = rbw;
        B.wcapr = st4[0];
        B.wcape = st4[1];
        B.RB = rbw;
        B.nrb = nrbw;
        B.nitems = (long long)P.G * nrbw;
        return 0;
    }
#ifndef FEAST_WIN_RB_MAX
#define FEAST_WIN_RB_MAX 80  // largest rows per staged item tried (80 complex FP32 only, 64, 32)
#endif
    for (const int rbw : {80, 64, 32}) {
        if (rbw > FEAST_WIN_RB_MAX || (rbw == 80 && P.fp64)) continue;
        int st4[4] = {0, 0, 0, 0};
        CK(cudaMemsetAsync(B.wstat, 0, sizeof(st4), s));
        CK(launch_win_build(P.n, rbw, B.app, B.apk, P.fp64, B.wpk, B.whdr, B.wwin, B.wstat, s));
        CK(cudaMemcpyAsync(st4, B.wstat, sizeof(st4), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (st4[3]) return 0;  // column indices outside [0, n): leave the matrix to the general path
        if (st4[2]) continue;
        const int nrbw = (P.n + rbw - 1) / rbw;
        if ((long long)P.G * nrbw >= (1ll << 31)) continue;  // items counted in 32-bit ints
        const size_t smem = win_smem_bytes(P.fp64, P.W, rbw, st4[0], st4[1]);
        const int occ = std::min(4, win_occupancy(P.fp64, P.W, B.bmode, rbw, smem));
        if (occ < 2) continue;
        B.wsmem = smem;
        B.wgrid = std::min(num_sms() * occ, nrbw);
        B.wrb = rbw;
        B.wcapr = st4[0];
        B.wcape = st4[1];
        B.RB = rbw;
        B.nrb = nrbw;
        B.nitems = (long long)P.G * nrbw;
        return 0;
    }
    return 0;
}

int setup_filter(const Plan& P, Bufs& B, const Csr& A, const Csr& Bm, const std::vector<double>& zw,
                 const double* lam, const int* mk, cudaStream_t s)
{
    CK(cudaMemcpyAsync(B.zw, zw.data(), sizeof(double) * zw.size(), cudaMemcpyHostToDevice, s));
    int amode = 0;
    int st = pack_matrix(A, P.fp64, false, B.app, B.apk, nullptr, &amode, s);
    if (st) return st;
    B.bmode = 0;
    if (P.hasB) {
        st = pack_matrix(Bm, P.fp64, true, B.bpp, B.bpk, B.bd, &B.bmode, s);
        if (st) return st;
    }
    st = choose_step_a(P, B, s);
    if (st) return st;
    FiltProb fp;
    memset(&fp, 0, sizeof(fp));
    fp.n = P.n;
    fp.m0 = P.m0;
    fp.G = P.G;
    fp.nrb = B.nrb;
    fp.item0 = 0;
    fp.nrb_b = P.nrb_b;
    fp.item0_b = 0;
    fp.vec_off = 0;
    fp.col_off = 0;
    fp.grp_off = 0;
    fp.q_off = 0;
    fp.dq_off = 0;
    fp.ia = A.ia;
    fp.ja = A.ja;
    fp.av = A.v;
    fp.ib = P.hasB ? Bm.ia : nullptr;
    fp.jb = P.hasB ? Bm.ja : nullptr;
    fp.bv = P.hasB ? Bm.v : nullptr;
    fp.app = B.app;
    fp.apk = B.apk;
    fp.bpp = B.bmode == 2 ? B.bpp : nullptr;
    fp.bpk = B.bmode == 2 ? B.bpk : nullptr;
    fp.bd = B.bmode == 1 ? B.bd : nullptr;
    fp.zw = B.zw;
    fp.lam = lam;
    fp.mk = mk;
    fp.ne = P.ne;
    fp.active = 1;
    CK(cudaMemcpyAsync(B.probs, &fp, sizeof(fp), cudaMemcpyHostToDevice, s));
    // the host copy of fp goes out of scope: make the upload complete first
    CK(cudaStreamSynchronize(s));
    return 0;
}

void log_line(int lvl, const char* text)
{
    if (lvl == 0) return;
    if (lvl > 0) {
        fputs(text, stdout);
        fflush(stdout);
        return;
    }
    char name[64];
    snprintf(name, sizeof(name), "feast%d.log", -lvl);
    FILE* f = fopen(name, "a");
    if (f) {
        fputs(text, f);
        fclose(f);
    }
}

// The FEAST iteration on device data.  x_dev: column-major n x m0 in/out.
int run_feast(const Plan& P, Bufs& B, const Csr& A, const Csr& Bm, int* fpm, double emin, double emax, int* m0io,
              double* e_host, double* x_dev, int* M_out, double* res_host, double* epsout, int* loop_out,
              cudaStream_t s, const double* custom_zw = nullptr)
{
    const int n = P.n, m0 = P.m0, ne = P.ne;
    const double alpha = std::max(std::fabs(emin), std::fabs(emax));
    const double eps = std::pow(10.0, -fpm[2]);
    const double tol = std::pow(10.0, -fpm[44]);
    const int maxit = fpm[45], maxloop = fpm[3];
    std::vector<double> zw;
    if (custom_zw) zw.assign(custom_zw, custom_zw + 4 * (size_t)ne);  // the caller's nodes (expert entry points)
    else contour(fpm[15], ne, emin, emax, fpm[17] / 100.0, zw);
    int st = setup_filter(P, B, A, Bm, zw, B.lam, B.mk, s);
    if (st) return st;
    // every subspace column is live until a reduced solve drops some
    CK(cudaMemcpyAsync(B.mk, &m0, sizeof(int), cudaMemcpyHostToDevice, s));
    const size_t blk = (size_t)n * m0;
    // start block Y (row-major) and the first right-hand side B Y
    if (fpm[4] == 1) {
        k_col_to_row<<<grid_for(blk), 256, 0, s>>>(n, m0, x_dev, B.Y);
        count_launches(1);
    } else {
        const unsigned long long seed = fpm[51] ? (unsigned long long)fpm[51] : 0x5EEDull;
        k_random_block<<<grid_for(blk), 256, 0, s>>>((long long)blk, seed, B.Y);
        count_launches(1);
    }
    CK(cudaGetLastError());
    size_t ph0 = 0;
    const int mode14 = fpm[13];  // 1: return the filtered block, 2: stochastic count
    if (fpm[4] == 1 && mode14 == 0) {
        // a given subspace is tested by Rayleigh-Ritz before any filtering, so
        // a converged subspace (e.g. a previous solution) returns at loop 0
        CK(cudaMemcpyAsync(B.Q, B.Y, sizeof(double) * blk, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(B.iter_max, 0, sizeof(int) * P.nbatch, s));
    } else {
        double* R = B.Y;
        if (P.hasB) {
            CK(launch_spmm_f64(n, m0, Bm.ia, Bm.ja, Bm.v, B.Y, B.T, s));
            R = B.T;
        }
        ph0 = g_prof.on ? g_prof.mark(s) : 0;
        st = filter_pass(P, B, 0, R, nullptr, maxit, tol, s);
        if (st) return st;
        if (g_prof.on) g_prof.phase.push_back({0, {ph0, g_prof.mark(s)}});
    }
    std::vector<int> itmax(P.nbatch);
    long long total_iters = 0;
    CK(cudaMemcpyAsync(itmax.data(), B.iter_max, sizeof(int) * P.nbatch, cudaMemcpyDeviceToHost, s));
    if (mode14 != 0) {
        // one contour pass only (fpm(14) = 1 or 2): no Rayleigh-Ritz
        CK(cudaStreamSynchronize(s));
        for (int b = 0; b < P.nbatch; ++b) total_iters += itmax[b];
        fpm[59] = (int)std::min<long long>(total_iters, 2147483647LL);
        for (int c = 0; c < m0; ++c) { e_host[c] = 0.0; res_host[c] = 0.0; }
        *M_out = 0;
        *loop_out = 0;
        *epsout = 0.0;
        if (mode14 == 1) {
            // the filtered block Q, column-major, into X (guide info 4)
            std::vector<int> id(m0);
            for (int c = 0; c < m0; ++c) id[c] = c;
            CK(cudaMemcpyAsync(B.perm, id.data(), sizeof(int) * m0, cudaMemcpyHostToDevice, s));
            k_gather_cols<<<grid_for(blk), 256, 0, s>>>(n, m0, m0, B.Q, B.perm, x_dev);
            count_launches(1);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(s));
            return 4;
        }
        // stochastic count (guide info 5): the probes are the columns of Y
        // (E[y y^T] = I), Q = rho(B^{-1}A) Y, and the mean of y_j^T Q_j
        // estimates trace(rho(B^{-1}A)), the number of eigenvalues inside
        CK(launch_coldot_f64(n, m0, B.Y, B.Q, B.rpart, B.res, s));
        std::vector<double> t(m0);
        CK(cudaMemcpyAsync(t.data(), B.res, sizeof(double) * m0, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double sum = 0.0, sum2 = 0.0;
        for (int c = 0; c < m0; ++c) {
            sum += t[c];
            sum2 += t[c] * t[c];
        }
        const double mean = sum / m0;
        const double var = m0 > 1 ? (sum2 - m0 * mean * mean) / (m0 - 1) : 0.0;
        e_host[0] = mean;
        if (m0 > 1) e_host[1] = std::sqrt(std::max(var, 0.0) / m0);
        *M_out = (int)std::max(0.0, std::floor(mean + 0.5));
        return 5;
    }

    std::vector<double> lam(m0), res(m0);
    int mk = m0, M = 0, info = 0, k = 0;
    double trace_prev = 0.0, eo = 1.0;
    char line[256];
    snprintf(line, sizeof(line), "#It |  #Eig  |          Trace            |     Error-Trace          |     Max-Residual\n");
    log_line(fpm[0], line);
    for (k = 0;; ++k) {
        // Rayleigh-Ritz on Q
        if (g_prof.on) ph0 = g_prof.mark(s);
        CK(launch_spmm_f64(n, m0, A.ia, A.ja, A.v, B.Q, B.T, s));
        auto gram = [&](const double* Xg, const double* Yg, double* Cg) {
            return P.oz ? launch_gram_oz(n, m0, Xg, Yg, Cg, B.gpart, B.ozex, s)
                        : launch_gram_f64(n, m0, Xg, Yg, Cg, B.gpart, P.ksplit, 1, s);
        };
        CK(gram(B.Q, B.T, B.Aq));
        if (P.hasB) {
            CK(launch_spmm_f64(n, m0, Bm.ia, Bm.ja, Bm.v, B.Q, B.T2, s));
            CK(gram(B.Q, B.T2, B.Bq));
        } else {
            CK(gram(B.Q, B.Q, B.Bq));
        }
        for (int b = 0; b < P.nbatch; ++b) total_iters += itmax[b];
        size_t ph1 = 0, ph2 = 0;
        if (g_prof.on) ph1 = g_prof.mark(s);
        const int rst = reduced_gev_dev(m0, B.Aq, B.Bq, B.lam, B.Vr, B.mk, B.eig, s);
        if (rst == -4) return cuda_fail(cudaGetLastError(), "reduced eigensolver");
        if (rst) { info = -3; break; }
        if (g_prof.on) ph2 = g_prof.mark(s);
        if (P.oz) CK(launch_gemm_oz(n, m0, m0, B.Q, B.Vr, B.X, B.ozw, s));
        else CK(launch_gemm_nn_f64(n, m0, m0, B.Q, B.Vr, B.X, s));
        CK(launch_residual_f64(n, m0, A.ia, A.ja, A.v, P.hasB ? Bm.ia : nullptr, P.hasB ? Bm.ja : nullptr,
                               P.hasB ? Bm.v : nullptr, B.X, B.lam, B.Y, B.rpart, nullptr, B.res, alpha, s));
        if (g_prof.on) {
            const size_t ph3 = g_prof.mark(s);
            g_prof.phase.push_back({1, {ph0, ph1}});
            g_prof.phase.push_back({2, {ph1, ph2}});
            g_prof.phase.push_back({3, {ph2, ph3}});
        }
        CK(cudaMemcpyAsync(lam.data(), B.lam, sizeof(double) * m0, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(res.data(), B.res, sizeof(double) * m0, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&mk, B.mk, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (mk < 1) { info = -3; break; }
        M = 0;
        double trace = 0.0, maxres = 0.0;
        for (int j = 0; j < mk; ++j)
            if (lam[j] >= emin && lam[j] <= emax) {
                ++M;
                trace += lam[j];
                maxres = std::max(maxres, res[j]);
            }
        eo = k == 0 ? 1.0 : std::fabs(trace - trace_prev) / alpha;
        trace_prev = trace;
        snprintf(line, sizeof(line), "%3d  %6d      %.16E      %.16E      %.16E\n", k, M, trace, eo,
                 M ? maxres : 1.0);
        log_line(fpm[0], line);
        const bool conv = M >= 1 && (fpm[5] == 1 ? maxres < eps : (k >= 1 && eo < eps));
        if (conv) { info = 0; break; }
        if (M == 0 && k >= 1) { info = 1; break; }
        if (k >= maxloop) { info = 2; break; }
        if (g_prof.on) ph0 = g_prof.mark(s);
        st = filter_pass(P, B, 1, B.Y, B.X, maxit, tol, s);
        if (st) return st;
        if (g_prof.on) g_prof.phase.push_back({0, {ph0, g_prof.mark(s)}});
        CK(cudaMemcpyAsync(itmax.data(), B.iter_max, sizeof(int) * P.nbatch, cudaMemcpyDeviceToHost, s));
    }
    fpm[59] = (int)std::min<long long>(total_iters, 2147483647LL);
    if (info == 0 && M >= mk) info = 3;
    // output order: inside ascending, then outside ascending
    std::vector<int> perm;
    if (info != -3) {
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < mk; ++j) {
                const bool in = lam[j] >= emin && lam[j] <= emax;
                if ((pass == 0) == in) perm.push_back(j);
            }
        for (int c = 0; c < mk; ++c) {
            e_host[c] = lam[perm[c]];
            res_host[c] = res[perm[c]];
        }
        for (int c = mk; c < m0; ++c) { e_host[c] = 0.0; res_host[c] = 0.0; }
        perm.resize(m0, 0);
        CK(cudaMemcpyAsync(B.perm, perm.data(), sizeof(int) * m0, cudaMemcpyHostToDevice, s));
        k_gather_cols<<<grid_for(blk), 256, 0, s>>>(n, m0, mk, B.X, B.perm, x_dev);
        count_launches(1);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
        *m0io = mk;
    }
    *M_out = M;
    *loop_out = k;
    *epsout = eo;
    if (g_prof.on) {
        unsigned long long work = 0;
        CK(cudaMemcpyAsync(&work, B.work, sizeof(work), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double* o = g_prof.out;
        // totals over every solve since the entry point started (the extreme
        // search runs several): recomputed, not added to
        for (int i = 0; i < 15; ++i) o[i] = 0.0;
        for (auto& pr : g_prof.a) o[0] += g_prof.ms(pr.first, pr.second);
        for (auto& pr : g_prof.b) o[1] += g_prof.ms(pr.first, pr.second);
        o[2] = (double)g_prof.a.size();
        o[3] = (double)g_prof.b.size();
        o[4] = (double)work;
        for (auto& ph : g_prof.phase) o[5 + ph.first] += g_prof.ms(ph.second.first, ph.second.second);
        o[9] = (double)P.W;
        o[10] = (double)P.mt;
        o[11] = (double)P.n;
        o[12] = (double)cplx_bytes(P);
        o[13] = (double)P.G;
        o[14] = (double)k;
        o[16] = (double)B.RB;
        o[17] = B.wws ? 2.0 : (B.wrb ? 1.0 : 0.0);
        o[18] = (double)(B.wrb ? B.wgrid : 0);
        o[19] = (double)(B.wrb ? B.wcapr : 0);
    }
    return info;
}

}  // namespace

// ---------------------------------------------------------------- device driver
// ---------------------------------------------------------------- extreme-eigenvalue search (fpm(40) = -1 / +1)
static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }
static constexpr int kGershBlocks = 1024;

// Workspace beyond the solver's own: -A (largest mode), diag(B), Gershgorin
// partials and a flag.
static size_t extreme_extra_bytes(int n, int nnz_a)
{
    return al256((size_t)nnz_a * sizeof(double)) + al256((size_t)n * sizeof(double)) +
           al256(2 * kGershBlocks * sizeof(double)) + 512;
}

extern "C" size_t feast_scsr_workspace_bytes(int n, int nnz_a, int nnz_b, int m0, const int* fpm)
{
    if (n <= 0 || m0 <= 0 || !fpm) return 0;
    Plan P = make_plan(n, nnz_a, nnz_b, m0, fpm);
    Bufs B;
    const size_t base = carve(P, nullptr, B);
    return fpm[39] != 0 ? al256(base) + extreme_extra_bytes(n, nnz_a) : base;
}

// Smallest and largest Gershgorin bound over the rows (scaled by diag(scale)
// when given).  Synchronises the stream.
static int gersh_bounds(const int* ia, const int* ja, const double* v, int n, const double* scale, double* part,
                        cudaStream_t s, double* lo, double* hi)
{
    const int blocks = std::max(1, std::min(kGershBlocks, (n + 255) / 256));
    k_gersh<<<blocks, 256, 0, s>>>(n, ia, ja, v, scale, part);
    count_launches(1);
    CK(cudaGetLastError());
    std::vector<double> h(2 * (size_t)blocks);
    CK(cudaMemcpyAsync(h.data(), part, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *lo = INFINITY;
    *hi = -INFINITY;
    for (int b = 0; b < blocks; ++b) {
        *lo = std::min(*lo, h[2 * b]);
        *hi = std::max(*hi, h[2 * b + 1]);
    }
    return 0;
}

// Bounds [lo, hi] of the spectrum of the pencil (A, B): Gershgorin discs of A
// (B = I), of D^{-1/2} A D^{-1/2} (B = D diagonal), or, for a general B whose
// Gershgorin interval is [bl, bu] with bl > 0, the bounds of the quotient
// x^T A x / x^T B x from A's interval [al, au]: [min(al/bl, al/bu),
// max(au/bl, au/bu)].  Returns 0, 7 when B cannot be shown positive definite
// this way, -4 on a CUDA error.
static int pencil_bounds(const Csr& A, const Csr& Bm, double* bdiag, int* flag, double* part, cudaStream_t s,
                         double* lo, double* hi)
{
    const int n = A.n;
    if (!Bm.v) return gersh_bounds(A.ia, A.ja, A.v, n, nullptr, part, s, lo, hi);
    CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
    k_csr_diag<<<grid_for(n), 256, 0, s>>>(n, Bm.ia, Bm.ja, Bm.v, bdiag, flag);
    count_launches(1);
    CK(cudaGetLastError());
    int offdiag = 0;
    CK(cudaMemcpyAsync(&offdiag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    double bl = 0.0, bu = 0.0;
    int r = gersh_bounds(Bm.ia, Bm.ja, Bm.v, n, nullptr, part, s, &bl, &bu);  // synchronises
    if (r) return r;
    if (!(bl > 0.0)) return 7;
    if (!offdiag) return gersh_bounds(A.ia, A.ja, A.v, n, bdiag, part, s, lo, hi);
    double al = 0.0, au = 0.0;
    r = gersh_bounds(A.ia, A.ja, A.v, n, nullptr, part, s, &al, &au);
    if (r) return r;
    *lo = std::min(al / bl, al / bu);
    *hi = std::max(au / bl, au / bu);
    return 0;
}

// The k = M0/2 lowest eigenpairs of (A, B) (fpm(40) = -1), or the k largest
// (fpm(40) = +1, the lowest of (-A, B) with the signs turned back).
//  1. Emin just below the Gershgorin lower bound of the pencil.
//  2. Emax by a search on the stochastic count (fpm(14) = 2 machinery, up to
//     32 seeded probes, the solver's contour settings) for an interval that
//     holds between 1.15 k and 1.5 k eigenvalues: grow the interval until the
//     count passes 1.15 k, then interpolate a power law count ~ span^p
//     between the bracketing spans (bisection of the log span as a fallback).
//  3. A normal solve on [Emin, Emax] with M0 = 2k; if it finds fewer than k
//     eigenvalues inside the interval grows by 35 %, if the subspace is too
//     small it shrinks by 20 %, each retry starting from the Ritz vectors just
//     found.
//  4. Output: M = k, E[0..k-1] the wanted eigenvalues ascending, the other
//     Ritz values after them, and the interval [emin, emax] that holds
//     exactly the k wanted eigenvalues (emax midway between the k-th and the
//     next Ritz value inside the searched interval when one was found).
// Returns the solver's info (0, or 2 when the last solve did not converge),
// 7 when no suitable interval was found, or an error code.
static int extreme_solve(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                         const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double* emin_io,
                         double* emax_io, int* m0, double* e, double* d_x, int* m, double* res, double* epsout,
                         int* loop, void* d_work, size_t work_bytes, cudaStream_t s)
{
    const int M0 = *m0, k = M0 / 2, sign = fpm[39];
    Plan Pm = make_plan(n, nnz_a, d_b ? nnz_b : 0, M0, fpm);
    Bufs Bw;
    const size_t need = carve(Pm, nullptr, Bw);
    if (!d_work || work_bytes < al256(need) + extreme_extra_bytes(n, nnz_a)) return -120;
    char* xp = (char*)d_work + al256(need);
    double* negA = (double*)xp;
    xp += al256((size_t)nnz_a * sizeof(double));
    double* bdiag = (double*)xp;
    xp += al256((size_t)n * sizeof(double));
    double* part = (double*)xp;
    xp += al256(2 * kGershBlocks * sizeof(double));
    int* flag = (int*)xp;
    const double* av = d_a;
    if (sign > 0) {
        k_negate<<<grid_for(nnz_a), 256, 0, s>>>(nnz_a, d_a, negA);
        count_launches(1);
        CK(cudaGetLastError());
        av = negA;
    }
    Csr A{n, nnz_a, d_ia, d_ja, av}, Bm{n, d_b ? nnz_b : 0, d_ib, d_jb, d_b};
    double lo = 0.0, hi = 0.0;
    int r = pencil_bounds(A, Bm, bdiag, flag, part, s, &lo, &hi);
    if (r) return r;
    char line[256];
    const double width = std::max(hi - lo, 1e-9 * std::max(1.0, std::fabs(lo)));
    const double Emin = lo - 0.01 * width;
    const double span_max = hi + 0.01 * width - Emin;
    snprintf(line, sizeof(line), "extreme search: spectrum bounds [%.10E, %.10E], Emin %.10E\n", lo, hi, Emin);
    log_line(fpm[0], line);

    // ---- interval search on stochastic counts
    int fpc[64];
    memcpy(fpc, fpm, sizeof(fpc));
    fpc[13] = 2;
    fpc[4] = 0;
    fpc[39] = 0;
    fpc[0] = 0;
    const int sp = std::max(2, std::min(M0, 32));
    const Plan Pc = make_plan(n, nnz_a, Bm.nnz, sp, fpc);
    auto count = [&](double E, double* est) -> int {
        Bufs Bc;
        carve(Pc, d_work, Bc);
        int mm = sp, Mi = 0, lp = 0;
        double eo = 0.0;
        std::vector<double> et(sp), rt(sp);
        CK(cudaMemsetAsync(Bc.work, 0, sizeof(unsigned long long), s));
        const int rr = run_feast(Pc, Bc, A, Bm, fpc, Emin, E, &mm, et.data(), d_x, &Mi, rt.data(), &eo, &lp, s);
        if (rr != 5) return rr < 0 ? rr : -2;
        *est = et[0];
        return 0;
    };
    const double t_lo = 1.15 * k, t_hi = 1.5 * k, t_mid = 1.3 * k;
    double d = std::min(span_max, width * std::min(1.0, t_mid / n));
    double dl = 0.0, nl = 0.0, dh = 0.0, nh = 0.0;
    bool have_l = false, have_h = false, found = false;
    for (int it = 0; it < 40; ++it) {
        d = std::min(d, span_max);
        double nu = 0.0;
        r = count(Emin + d, &nu);
        if (r) return r;
        snprintf(line, sizeof(line), "extreme search: Emax %.10E  estimated count %.2f\n", Emin + d, nu);
        log_line(fpm[0], line);
        if ((nu >= t_lo && nu <= t_hi) || (nu < t_lo && d >= span_max)) {
            found = true;
            break;
        }
        if (nu < t_lo) { dl = d; nl = nu; have_l = true; }
        else { dh = d; nh = nu; have_h = true; }
        double dn;
        if (!have_h) dn = d * std::min(8.0, std::max(1.25, nu > 0.5 ? t_mid / nu : 8.0));
        else if (!have_l) dn = d * std::max(0.125, std::min(0.8, t_mid / nu));
        else {
            dn = std::sqrt(dl * dh);
            if (nl > 0.5) {
                const double pw = std::log(nh / nl) / std::log(dh / dl);
                const double di = dl * std::pow(t_mid / nl, 1.0 / pw);
                if (pw > 0.0 && di > dl && di < dh) dn = di;
            }
        }
        d = dn;
    }
    if (!found) return 7;
    double E = Emin + d;

    // ---- solves on [Emin, E]
    int fps[64];
    memcpy(fps, fpm, sizeof(fps));
    fps[39] = 0;
    fps[13] = 0;
    int info = 7, mk = M0;
    for (int attempt = 0; attempt < 5; ++attempt) {
        carve(Pm, d_work, Bw);
        CK(cudaMemsetAsync(Bw.work, 0, sizeof(unsigned long long), s));
        mk = M0;
        r = run_feast(Pm, Bw, A, Bm, fps, Emin, E, &mk, e, d_x, m, res, epsout, loop, s);
        if (r < 0) return r;
        snprintf(line, sizeof(line), "extreme search: solve on [%.10E, %.10E]: info %d, %d inside\n", Emin, E, r, *m);
        log_line(fpm[0], line);
        if ((r == 0 || r == 2) && *m >= k) {
            info = r;
            break;
        }
        if (r == 3) E = Emin + 0.8 * (E - Emin);
        else E = Emin + 1.35 * (E - Emin);
        fps[4] = 1;  // start again from the Ritz vectors just found
    }
    fpm[59] = fps[59];
    *m0 = mk;
    if (info == 7) return 7;
    const double Eout = *m > k ? 0.5 * (e[k - 1] + e[k]) : E;
    *m = k;
    if (sign > 0) {
        for (int c = 0; c < mk; ++c) e[c] = -e[c];
        std::reverse(e, e + k);
        std::reverse(res, res + k);
        std::reverse(e + k, e + mk);
        std::reverse(res + k, res + mk);
        k_reverse_cols<<<grid_for((long long)n * k), 256, 0, s>>>(n, 0, k, d_x);
        k_reverse_cols<<<grid_for((long long)n * (mk - k + 1)), 256, 0, s>>>(n, k, mk, d_x);
        count_launches(2);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
        *emin_io = -Eout;
        *emax_io = -Emin;
    } else {
        *emin_io = Emin;
        *emax_io = Eout;
    }
    return info;
}

extern "C" int feast_scsr_extreme_dev(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a,
                                      int nnz_b, const int* d_ib, const int* d_jb, const double* d_b, int* fpm,
                                      double* emin, double* emax, int* m0, double* e, double* d_x, int* m,
                                      double* res, double* epsout, int* loop, int* info, void* d_work,
                                      size_t work_bytes, void* stream)
{
    int inf = 0;
    auto ret = [&](int v) { if (info) *info = v; return v; };
    if (!fpm) return ret(-109);
    if (n <= 0) return ret(202);
    if (!m0 || *m0 < 2 || *m0 > n) return ret(201);
    if ((inf = check_fpm(fpm))) return ret(inf);
    if (fpm[39] != -1 && fpm[39] != 1) return ret(140);
    if (fpm[13] != 0) return ret(114);
    if (!d_ia || !d_ja || !d_a || nnz_a < 0) return ret(-103);
    if (d_b && (!d_ib || !d_jb || nnz_b <= 0)) return ret(-106);
    if (!emin) return ret(-110);
    if (!emax) return ret(-111);
    if (!e || !d_x || !m || !res || !epsout || !loop) return ret(-113);
    g_err.clear();
    g_prof.reset(fpm[52] == 1);
    const long long l0 = launch_count();
    inf = extreme_solve(n, nnz_a, d_ia, d_ja, d_a, nnz_b, d_ib, d_jb, d_b, fpm, emin, emax, m0, e, d_x, m, res,
                        epsout, loop, d_work, work_bytes, (cudaStream_t)stream);
    g_prof.out[15] = (double)(launch_count() - l0);
    return ret(inf);
}

// Custom nodes (expert entry points): z, w host arrays of 2 ne doubles (re,
// im) in the convention of feast_contour_nodes; every node strictly in the
// upper half plane and finite.  Returns 0 and fills zw (z.re, z.im, w.re,
// w.im per node), or the given error code.
static int custom_nodes(int ne, const double* z, const double* w, int bad, std::vector<double>& zw)
{
    if (!z || !w) return bad;
    zw.assign(4 * (size_t)ne, 0.0);
    for (int e = 0; e < ne; ++e) {
        if (!(z[2 * e + 1] > 0.0) || !std::isfinite(z[2 * e]) || !std::isfinite(z[2 * e + 1]) ||
            !std::isfinite(w[2 * e]) || !std::isfinite(w[2 * e + 1]))
            return bad;
        zw[4 * e] = z[2 * e];
        zw[4 * e + 1] = z[2 * e + 1];
        zw[4 * e + 2] = w[2 * e];
        zw[4 * e + 3] = w[2 * e + 1];
    }
    return 0;
}

static int solve_dev_impl(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                          const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double emin, double emax,
                          int* m0, double* e, double* d_x, int* m, double* res, double* epsout, int* loop,
                          int* info, void* d_work, size_t work_bytes, void* stream, const double* zne,
                          const double* wne, bool expert);

extern "C" int feast_scsr_solve_dev(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a,
                                    int nnz_b, const int* d_ib, const int* d_jb, const double* d_b, int* fpm,
                                    double emin, double emax, int* m0, double* e, double* d_x, int* m,
                                    double* res, double* epsout, int* loop, int* info, void* d_work,
                                    size_t work_bytes, void* stream)
{
    return solve_dev_impl(n, nnz_a, d_ia, d_ja, d_a, nnz_b, d_ib, d_jb, d_b, fpm, emin, emax, m0, e, d_x, m, res,
                          epsout, loop, info, d_work, work_bytes, stream, nullptr, nullptr, false);
}

extern "C" int feast_scsr_solve_dev_x(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a,
                                      int nnz_b, const int* d_ib, const int* d_jb, const double* d_b, int* fpm,
                                      double emin, double emax, int* m0, double* e, double* d_x, int* m,
                                      double* res, double* epsout, int* loop, int* info, void* d_work,
                                      size_t work_bytes, void* stream, const double* zne, const double* wne)
{
    return solve_dev_impl(n, nnz_a, d_ia, d_ja, d_a, nnz_b, d_ib, d_jb, d_b, fpm, emin, emax, m0, e, d_x, m, res,
                          epsout, loop, info, d_work, work_bytes, stream, zne, wne, true);
}

static int solve_dev_impl(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                          const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double emin, double emax,
                          int* m0, double* e, double* d_x, int* m, double* res, double* epsout, int* loop,
                          int* info, void* d_work, size_t work_bytes, void* stream, const double* zne,
                          const double* wne, bool expert)
{
    int inf = 0;
    auto ret = [&](int v) { if (info) *info = v; return v; };
    if (!fpm) return ret(-109);
    if (n <= 0) return ret(202);
    if (!m0 || *m0 <= 0 || *m0 > n) return ret(201);
    if (!(emin < emax)) return ret(200);
    if ((inf = check_fpm(fpm))) return ret(inf);
    if (fpm[39] != 0) return ret(140);  // extreme-eigenvalue search: feast_scsr_extreme_dev
    if (!d_ia || !d_ja || !d_a || nnz_a < 0) return ret(-103);
    if (d_b && (!d_ib || !d_jb || nnz_b <= 0)) return ret(-106);
    if (!e || !d_x || !m || !res || !epsout || !loop) return ret(-113);
    Plan P = make_plan(n, nnz_a, d_b ? nnz_b : 0, *m0, fpm);
    Bufs B;
    const size_t need = carve(P, nullptr, B);
    if (!d_work || work_bytes < need) return ret(-120);
    std::vector<double> czw;
    if (expert && (inf = custom_nodes(fpm[1], zne, wne, -124, czw))) return ret(inf);
    carve(P, d_work, B);
    Csr A{n, nnz_a, d_ia, d_ja, d_a}, Bm{n, d_b ? nnz_b : 0, d_ib, d_jb, d_b};
    g_err.clear();
    g_prof.reset(fpm[52] == 1);
    const long long l0 = launch_count();
    CK(cudaMemsetAsync(B.work, 0, sizeof(unsigned long long), (cudaStream_t)stream));
    inf = run_feast(P, B, A, Bm, fpm, emin, emax, m0, e, d_x, m, res, epsout, loop, (cudaStream_t)stream,
                    expert ? czw.data() : nullptr);
    g_prof.out[15] = (double)(launch_count() - l0);
    return ret(inf);
}

// ---------------------------------------------------------------- host driver
namespace {

// Validate a host CSR (base = ia[0] in {0,1}) and expand it to 0-based full
// storage.  Returns 0 or the argument's error code.
int host_csr(char uplo, int n, const double* v, const int* ia, const int* ja, int arg0, std::vector<int>& oia,
             std::vector<int>& oja, std::vector<double>& ov)
{
    if (!v) return -(100 + arg0);
    if (!ia) return -(100 + arg0 + 1);
    if (!ja) return -(100 + arg0 + 2);
    const int base = ia[0];
    if (base != 0 && base != 1) return -(100 + arg0 + 1);
    for (int i = 0; i < n; ++i)
        if (ia[i + 1] < ia[i]) return -(100 + arg0 + 1);
    const long long nnz = (long long)ia[n] - base;
    if (uplo == 'F') {  // full storage: validate and copy in one pass while the rows are sorted
        oia.resize((size_t)n + 1);
        oja.resize((size_t)nnz);
        ov.resize((size_t)nnz);
        bool sorted = true;
        for (int i = 0; i <= n; ++i) oia[i] = ia[i] - base;
        for (int i = 0; i < n && sorted; ++i) {
            int prev = -1;
            for (int p = oia[i]; p < oia[i + 1]; ++p) {
                const int j = ja[p] - base;
                if (j < 0 || j >= n) return -(100 + arg0 + 2);
                if (!std::isfinite(v[p])) return -(100 + arg0);
                if (j <= prev) { sorted = false; break; }  // unsorted or repeated: general path below
                prev = j;
                oja[p] = j;
                ov[p] = v[p];
            }
        }
        if (sorted) return 0;
    }
    std::vector<std::vector<std::pair<int, double>>> rows(n);
    for (int i = 0; i < n; ++i)
        for (int p = ia[i] - base; p < ia[i + 1] - base; ++p) {
            const int j = ja[p] - base;
            if (j < 0 || j >= n) return -(100 + arg0 + 2);
            if (!std::isfinite(v[p])) return -(100 + arg0);
            if (uplo == 'L' && j > i) return -(100 + arg0 + 2);
            if (uplo == 'U' && j < i) return -(100 + arg0 + 2);
            rows[i].push_back({j, v[p]});
            if (uplo != 'F' && j != i) rows[j].push_back({i, v[p]});
        }
    (void)nnz;
    oia.assign(n + 1, 0);
    oja.clear();
    ov.clear();
    for (int i = 0; i < n; ++i) {
        std::sort(rows[i].begin(), rows[i].end(),
                  [](const std::pair<int, double>& a, const std::pair<int, double>& b) { return a.first < b.first; });
        for (auto& pr : rows[i]) {
            oja.push_back(pr.first);
            ov.push_back(pr.second);
        }
        oia[i + 1] = (int)oja.size();
    }
    return 0;
}

struct DevMem {
    std::vector<void*> ptrs;
    ~DevMem()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t count)
    {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 256);
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            *p = (T*)q;
        }
        return e;
    }
};

}  // namespace

// Host-memory driver shared by feast_scsr_solve (extreme = false: the
// interval is an input) and feast_scsr_extreme (the interval is found and
// returned): validates and expands the CSR, copies it to the device, runs the
// device entry point and copies X back.
static int host_driver(bool extreme, char uplo, int n, const double* a, const int* ia, const int* ja,
                       const double* b, const int* ib, const int* jb, int* fpm, double* emin_io, double* emax_io,
                       int* m0, double* e, double* x, int* m, double* res, double* epsout, int* loop, int* info,
                       const double* zne = nullptr, const double* wne = nullptr, bool expert = false)
{
    auto ret = [&](int v) { if (info) *info = v; return v; };
    if (uplo != 'F' && uplo != 'L' && uplo != 'U') return ret(-101);
    if (n <= 0) return ret(202);
    if (!fpm) return ret(-109);
    int inf = check_fpm(fpm);
    if (inf) return ret(inf);
    if (!extreme && fpm[39] != 0) return ret(140);  // extreme-eigenvalue search: feast_scsr_extreme
    if (extreme && fpm[39] != -1 && fpm[39] != 1) return ret(140);
    if (extreme && fpm[13] != 0) return ret(114);
    if (!extreme && !(*emin_io < *emax_io)) return ret(200);
    if (expert) {
        std::vector<double> czw;
        if ((inf = custom_nodes(fpm[1], zne, wne, -120, czw))) return ret(inf);
    }
    if (!m0 || *m0 <= (extreme ? 1 : 0) || *m0 > n) return ret(201);
    if (!e) return ret(-113);
    if (!x) return ret(-114);
    if (!m) return ret(-115);
    if (!res) return ret(-116);
    if (!epsout) return ret(-117);
    if (!loop) return ret(-118);
    std::vector<int> aia, aja, bia, bja;
    std::vector<double> av, bv;
    inf = host_csr(uplo, n, a, ia, ja, 3, aia, aja, av);
    if (inf) return ret(inf);
    const bool hasB = b || ib || jb;
    if (hasB) {
        inf = host_csr(uplo, n, b, ib, jb, 6, bia, bja, bv);
        if (inf) return ret(inf);
    }
    g_err.clear();
    const int mm0 = *m0;
    DevMem dm;
    int *d_ia = nullptr, *d_ja = nullptr, *d_ib = nullptr, *d_jb = nullptr;
    double *d_a = nullptr, *d_b = nullptr, *d_x = nullptr;
    void* d_work = nullptr;
    cudaStream_t s = nullptr;
    const size_t wb = feast_scsr_workspace_bytes(n, (int)aja.size(), hasB ? (int)bja.size() : 0, mm0, fpm);
#define HK(x)                                                        \
    do {                                                             \
        cudaError_t _e = (x);                                        \
        if (_e != cudaSuccess) return ret(cuda_fail(_e, #x));        \
    } while (0)
    HK(dm.alloc(&d_ia, aia.size()));
    HK(dm.alloc(&d_ja, std::max<size_t>(1, aja.size())));
    HK(dm.alloc(&d_a, std::max<size_t>(1, av.size())));
    HK(dm.alloc(&d_x, (size_t)n * mm0));
    HK(dm.alloc((char**)&d_work, wb));
    HK(cudaMemcpy(d_ia, aia.data(), sizeof(int) * aia.size(), cudaMemcpyHostToDevice));
    HK(cudaMemcpy(d_ja, aja.data(), sizeof(int) * aja.size(), cudaMemcpyHostToDevice));
    HK(cudaMemcpy(d_a, av.data(), sizeof(double) * av.size(), cudaMemcpyHostToDevice));
    if (hasB) {
        HK(dm.alloc(&d_ib, bia.size()));
        HK(dm.alloc(&d_jb, std::max<size_t>(1, bja.size())));
        HK(dm.alloc(&d_b, std::max<size_t>(1, bv.size())));
        HK(cudaMemcpy(d_ib, bia.data(), sizeof(int) * bia.size(), cudaMemcpyHostToDevice));
        HK(cudaMemcpy(d_jb, bja.data(), sizeof(int) * bja.size(), cudaMemcpyHostToDevice));
        HK(cudaMemcpy(d_b, bv.data(), sizeof(double) * bv.size(), cudaMemcpyHostToDevice));
    }
    if (fpm[4] == 1) HK(cudaMemcpy(d_x, x, sizeof(double) * (size_t)n * mm0, cudaMemcpyHostToDevice));
    if (extreme)
        inf = feast_scsr_extreme_dev(n, (int)aja.size(), d_ia, d_ja, d_a, hasB ? (int)bja.size() : 0, d_ib, d_jb,
                                     d_b, fpm, emin_io, emax_io, m0, e, d_x, m, res, epsout, loop, info, d_work, wb, s);
    else
        inf = solve_dev_impl(n, (int)aja.size(), d_ia, d_ja, d_a, hasB ? (int)bja.size() : 0, d_ib, d_jb, d_b, fpm,
                             *emin_io, *emax_io, m0, e, d_x, m, res, epsout, loop, info, d_work, wb, s, zne, wne,
                             expert);
    if ((inf >= 0 && inf != 5) || inf == -3 || inf == -2)  // info 5 (count only) leaves X alone
        HK(cudaMemcpy(x, d_x, sizeof(double) * (size_t)n * mm0, cudaMemcpyDeviceToHost));
#undef HK
    return ret(inf);
}

extern "C" int feast_scsr_solve(char uplo, int n, const double* a, const int* ia, const int* ja, const double* b,
                                const int* ib, const int* jb, int* fpm, double emin, double emax, int* m0,
                                double* e, double* x, int* m, double* res, double* epsout, int* loop, int* info)
{
    return host_driver(false, uplo, n, a, ia, ja, b, ib, jb, fpm, &emin, &emax, m0, e, x, m, res, epsout, loop,
                       info);
}

extern "C" int feast_scsr_solve_x(char uplo, int n, const double* a, const int* ia, const int* ja, const double* b,
                                  const int* ib, const int* jb, int* fpm, double emin, double emax, int* m0,
                                  double* e, double* x, int* m, double* res, double* epsout, int* loop, int* info,
                                  const double* zne, const double* wne)
{
    return host_driver(false, uplo, n, a, ia, ja, b, ib, jb, fpm, &emin, &emax, m0, e, x, m, res, epsout, loop,
                       info, zne, wne, true);
}

extern "C" int feast_scsr_extreme(char uplo, int n, const double* a, const int* ia, const int* ja, const double* b,
                                  const int* ib, const int* jb, int* fpm, double* emin, double* emax, int* m0,
                                  double* e, double* x, int* m, double* res, double* epsout, int* loop, int* info)
{
    if (!emin) { if (info) *info = -110; return -110; }
    if (!emax) { if (info) *info = -111; return -111; }
    return host_driver(true, uplo, n, a, ia, ja, b, ib, jb, fpm, emin, emax, m0, e, x, m, res, epsout, loop, info);
}

// ---------------------------------------------------------------- kernel-level entry points
namespace {
struct AsyncMem {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit AsyncMem(cudaStream_t st) : s(st) {}
    ~AsyncMem()
    {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    cudaError_t alloc(void** p, size_t bytes)
    {
        cudaError_t e = cudaMallocAsync(p, bytes + 256, s);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};
}  // namespace

extern "C" int feast_shifted_spmm_dev(int n, int nnz_a, const int* ia, const int* ja, const double* a, int nnz_b,
                                      const int* ib, const int* jb, const double* b, int nb, const double* z, int m,
                                      int fp64, const void* P, void* V, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return -101;
    if (nb < 1 || nb > 32) return -110;
    if (m <= 0) return -112;
    int W, nbp, mt;
    feast_filter_layout(nb, fp64, &W, &nbp, &mt);
    const int G = (m + mt - 1) / mt;
    const int RB = 256;
    const int nrb = (n + RB - 1) / RB;
    std::vector<ColState> cs((size_t)G * W);
    memset(cs.data(), 0, sizeof(ColState) * cs.size());
    for (int c = 0; c < G * W; ++c) {
        const int e = (c % W) % nbp;
        if (e < nb) cs[c].z = make_double2(z[2 * e], z[2 * e + 1]);
    }
    AsyncMem am(s);
    void *d_cs = nullptr, *d_fp = nullptr, *apk = nullptr, *bpk = nullptr, *app = nullptr, *bpp = nullptr,
         *bd = nullptr;
    const size_t pk = fp64 ? 16 : 8;
    CK(am.alloc(&d_cs, sizeof(ColState) * cs.size()));
    CK(am.alloc(&d_fp, sizeof(FiltProb)));
    CK(am.alloc(&app, sizeof(int) * ((size_t)n + 1)));
    CK(am.alloc(&apk, pk * ((size_t)nnz_a + 7 * (size_t)n)));
    int amode = 0, bmode = 0;
    int st = pack_matrix(Csr{n, nnz_a, ia, ja, a}, fp64 != 0, false, (int*)app, apk, nullptr, &amode, s);
    if (st) return st;
    if (b) {
        CK(am.alloc(&bpp, sizeof(int) * ((size_t)n + 1)));
        CK(am.alloc(&bpk, pk * ((size_t)nnz_b + 7 * (size_t)n)));
        CK(am.alloc(&bd, sizeof(double) * (size_t)n));
        st = pack_matrix(Csr{n, nnz_b, ib, jb, b}, fp64 != 0, true, (int*)bpp, bpk, bd, &bmode, s);
        if (st) return st;
    }
    FiltProb fp;
    memset(&fp, 0, sizeof(fp));
    fp.n = n;
    fp.m0 = m;
    fp.G = G;
    fp.nrb = nrb;
    fp.ia = ia;
    fp.ja = ja;
    fp.av = a;
    fp.ib = b ? ib : nullptr;
    fp.jb = b ? jb : nullptr;
    fp.bv = b;
    fp.app = (const int*)app;
    fp.apk = apk;
    fp.bpp = bmode == 2 ? (const int*)bpp : nullptr;
    fp.bpk = bmode == 2 ? bpk : nullptr;
    fp.bd = bmode == 1 ? bd : nullptr;
    fp.active = 1;
    CK(cudaMemcpyAsync(d_cs, cs.data(), sizeof(ColState) * cs.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_fp, &fp, sizeof(fp), cudaMemcpyHostToDevice, s));
    FilterArgs fa;
    memset(&fa, 0, sizeof(fa));
    memset(&fa, 0, sizeof(fa));
    fa.probs = (const FiltProb*)d_fp;
    fa.nprob = 1;
    fa.nitems = (long long)G * nrb;
    fa.W = W;
    fa.nbp = nbp;
    fa.mt = mt;
    fa.RB = RB;
    fa.hasB = b ? 1 : 0;
    fa.bmode = bmode;
    fa.p0 = const_cast<void*>(P);
    fa.p1 = V;
    fa.cs = (ColState*)d_cs;
    const int grid = (int)std::min<long long>(filter_grid(fp64 != 0, W), fa.nitems);
    CK(launch_shifted_spmm(fa, fp64 != 0, grid, s));
    CK(cudaStreamSynchronize(s));
    return 0;
}

extern "C" int feast_filter_dev(int n, int nnz_a, const int* ia, const int* ja, const double* a, int nnz_b,
                                const int* ib, const int* jb, const double* b, int m, const double* R,
                                const double* X, const double* lam, int rii, const int* fpm, double emin,
                                double emax, double* Q, int* iters, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return -101;
    if (m <= 0 || m > n) return -110;
    if (!fpm) return -115;
    int inf = check_fpm(fpm);
    if (inf) return inf;
    if (!(emin < emax)) return 200;
    Plan P = make_plan(n, nnz_a, b ? nnz_b : 0, m, fpm, true);
    Bufs B;
    const size_t bytes = carve(P, nullptr, B, true);
    AsyncMem am(s);
    void* base = nullptr;
    CK(am.alloc(&base, bytes));
    carve(P, base, B, true);
    Csr A{n, nnz_a, ia, ja, a}, Bm{n, b ? nnz_b : 0, ib, jb, b};
    std::vector<double> zw;
    contour(fpm[15], P.ne, emin, emax, fpm[17] / 100.0, zw);
    int st = setup_filter(P, B, A, Bm, zw, lam, nullptr, s);
    if (st) return st;
    B.Q = Q;
    st = filter_pass(P, B, rii, R, X, fpm[45], std::pow(10.0, -fpm[44]), s);
    if (st) return st;
    std::vector<int> itm(P.nbatch);
    CK(cudaMemcpyAsync(itm.data(), B.iter_max, sizeof(int) * P.nbatch, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (iters) {
        int t = 0;
        for (int v : itm) t += v;
        *iters = t;
    }
    return 0;
}

extern "C" int feast_gram_dev(int n, int m, const double* X, const double* Y, double* C, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return -101;
    if (m <= 0) return -102;
    int ks = 1;
    const size_t gp = gram_partial_doubles(n, m, &ks, num_sms());
    AsyncMem am(s);
    void* part = nullptr;
    CK(am.alloc(&part, gp * sizeof(double)));
    CK(launch_gram_f64(n, m, X, Y, C, (double*)part, ks, 1, s));
    CK(cudaStreamSynchronize(s));
    return 0;
}

extern "C" int feast_gram_oz_dev(int n, int m, const double* X, const double* Y, double* C, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return -101;
    if (m <= 0) return -102;
    const size_t gp = gram_oz_partial_doubles(n, m, nullptr, nullptr, num_sms());
    AsyncMem am(s);
    void* part = nullptr;
    void* ex = nullptr;
    CK(am.alloc(&part, gp * sizeof(double)));
    CK(am.alloc(&ex, gram_oz_work_bytes(m)));
    CK(launch_gram_oz(n, m, X, Y, C, (double*)part, (int*)ex, s));
    CK(cudaStreamSynchronize(s));
    return 0;
}

extern "C" int feast_gemm_oz_dev(int n, int m, int k, const double* A, const double* V, double* C, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return -101;
    if (m <= 0) return -102;
    if (k <= 0) return -103;
    AsyncMem am(s);
    void* w = nullptr;
    CK(am.alloc(&w, gemm_oz_work_bytes(n, m, k)));
    CK(launch_gemm_oz(n, m, k, A, V, C, w, s));
    CK(cudaStreamSynchronize(s));
    return 0;
}

extern "C" int feast_gemm_dev(int n, int m, int k, const double* A, const double* V, double* C, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return -101;
    if (m <= 0) return -102;
    if (k <= 0) return -103;
    CK(launch_gemm_nn_f64(n, m, k, A, V, C, s));
    CK(cudaStreamSynchronize(s));
    return 0;
}

extern "C" int feast_sym_eig_dev(int m, double* A, double* lam, double* V, int* sweeps, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (m <= 0) return -101;
    AsyncMem am(s);
    void* w = nullptr;
    CK(am.alloc(&w, jacobi_work_bytes(m)));
    int sw = 0;
    const int st = jacobi_eig_dev(m, A, lam, V, w, s, &sw);
    if (sweeps) *sweeps = sw;
    if (st == -3) return cuda_fail(cudaGetLastError(), "jacobi");
    return st ? -3 : 0;
}

extern "C" int feast_reduced_eig_dev(int m, const double* Aq, const double* Bq, double* lam, double* V, int* mk,
                                     void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (m <= 0) return -101;
    AsyncMem am(s);
    void* w = nullptr;
    void* dmk = nullptr;
    CK(am.alloc(&w, reduced_work_bytes(m)));
    CK(am.alloc(&dmk, sizeof(int)));
    const int st = reduced_gev_dev(m, Aq, Bq, lam, V, (int*)dmk, w, s);
    if (st == -4) return cuda_fail(cudaGetLastError(), "reduced eigensolver");
    if (st) return -3;
    int h = 0;
    CK(cudaMemcpyAsync(&h, dmk, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (mk) *mk = h;
    return 0;
}

extern "C" int feast_residual_dev(int n, const int* ia, const int* ja, const double* a, const int* ib,
                                  const int* jb, const double* b, int m, const double* X, const double* lam,
                                  double alpha, double* R, double* res, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return -101;
    if (m <= 0) return -108;
    AsyncMem am(s);
    void* part = nullptr;
    CK(am.alloc(&part, residual_partial_doubles(n, m) * sizeof(double)));
    CK(launch_residual_f64(n, m, ia, ja, a, ib, jb, b, X, lam, R, (double*)part, nullptr, res, alpha, s));
    CK(cudaStreamSynchronize(s));
    return 0;
}

extern "C" int feast_eig_grad_dev(int n, const int* ia, const int* ja, int m, const double* X, const double* w,
                                  double* grad, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return -101;
    if (m <= 0 || m > 2048) return -104;
    CK(launch_eig_grad(n, ia, ja, m, X, w, grad, s));
    CK(cudaStreamSynchronize(s));
    return 0;
}

// Validate one host CSR pattern (base ia[0] in {0,1}, rows nondecreasing,
// columns in range and in the stored triangle for 'L'/'U') and make a 0-based
// copy.  arg0 is the argument number of ia.
static int host_pattern(char uplo, int n, const int* ia, const int* ja, int arg0, std::vector<int>& oia,
                        std::vector<int>& oja)
{
    if (!ia) return -(100 + arg0);
    if (!ja) return -(100 + arg0 + 1);
    const int base = ia[0];
    if (base != 0 && base != 1) return -(100 + arg0);
    for (int i = 0; i < n; ++i)
        if (ia[i + 1] < ia[i]) return -(100 + arg0);
    oia.resize(n + 1);
    for (int i = 0; i <= n; ++i) oia[i] = ia[i] - base;
    oja.resize(std::max(1, oia[n]));
    for (int i = 0; i < n; ++i)
        for (int p = oia[i]; p < oia[i + 1]; ++p) {
            const int j = ja[p] - base;
            if (j < 0 || j >= n) return -(100 + arg0 + 1);
            if ((uplo == 'L' && j > i) || (uplo == 'U' && j < i)) return -(100 + arg0 + 1);
            oja[p] = j;
        }
    return 0;
}

extern "C" int feast_scsr_grad(char uplo, int n, const int* ia, const int* ja, const int* ib, const int* jb, int m,
                               const double* x, const double* e, const double* g, double* grad_a, double* grad_b)
{
    if (uplo != 'F' && uplo != 'L' && uplo != 'U') return -101;
    if (n <= 0) return 202;
    const bool hasB = ib || jb;
    if (m < 0 || m > 2048) return -107;
    if (!x) return -108;
    if (hasB && !e) return -109;
    if (!g) return -110;
    if (!grad_a) return -111;
    if (hasB && !grad_b) return -112;
    std::vector<int> aia, aja, bia, bja;
    int inf = host_pattern(uplo, n, ia, ja, 3, aia, aja);
    if (inf) return inf;
    if (hasB && (inf = host_pattern(uplo, n, ib, jb, 5, bia, bja))) return inf;
    const int nnz_a = aia[n], nnz_b = hasB ? bia[n] : 0;
    if (m == 0) {
        for (int p = 0; p < nnz_a; ++p) grad_a[p] = 0.0;
        for (int p = 0; p < nnz_b; ++p) grad_b[p] = 0.0;
        return 0;
    }
    g_err.clear();
    DevMem dm;
    int *d_ia = nullptr, *d_ja = nullptr, *d_ib = nullptr, *d_jb = nullptr;
    double *d_xc = nullptr, *d_xr = nullptr, *d_g = nullptr, *d_e = nullptr, *d_ga = nullptr, *d_gb = nullptr;
    const int half = uplo != 'F';
#define GK(x)                                                  \
    do {                                                       \
        cudaError_t _e = (x);                                  \
        if (_e != cudaSuccess) return cuda_fail(_e, #x);       \
    } while (0)
    GK(dm.alloc(&d_ia, (size_t)n + 1));
    GK(dm.alloc(&d_ja, aja.size()));
    GK(dm.alloc(&d_xc, (size_t)n * m));
    GK(dm.alloc(&d_xr, (size_t)n * m));
    GK(dm.alloc(&d_g, (size_t)m));
    GK(dm.alloc(&d_ga, (size_t)std::max(1, nnz_a)));
    GK(cudaMemcpy(d_ia, aia.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    GK(cudaMemcpy(d_ja, aja.data(), sizeof(int) * aja.size(), cudaMemcpyHostToDevice));
    GK(cudaMemcpy(d_xc, x, sizeof(double) * (size_t)n * m, cudaMemcpyHostToDevice));
    GK(cudaMemcpy(d_g, g, sizeof(double) * m, cudaMemcpyHostToDevice));
    k_col_to_row<<<grid_for((long long)n * m), 256>>>(n, m, d_xc, d_xr);
    count_launches(1);
    GK(cudaGetLastError());
    GK(launch_eig_grad(n, d_ia, d_ja, m, d_xr, d_g, d_ga, nullptr, nullptr, half));
    if (hasB) {
        GK(dm.alloc(&d_ib, (size_t)n + 1));
        GK(dm.alloc(&d_jb, bja.size()));
        GK(dm.alloc(&d_e, (size_t)m));
        GK(dm.alloc(&d_gb, (size_t)std::max(1, nnz_b)));
        GK(cudaMemcpy(d_ib, bia.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
        GK(cudaMemcpy(d_jb, bja.data(), sizeof(int) * bja.size(), cudaMemcpyHostToDevice));
        GK(cudaMemcpy(d_e, e, sizeof(double) * m, cudaMemcpyHostToDevice));
        GK(launch_eig_grad(n, d_ib, d_jb, m, d_xr, d_g, d_gb, nullptr, d_e, half));
    }
    GK(cudaMemcpy(grad_a, d_ga, sizeof(double) * nnz_a, cudaMemcpyDeviceToHost));
    if (hasB) GK(cudaMemcpy(grad_b, d_gb, sizeof(double) * nnz_b, cudaMemcpyDeviceToHost));
#undef GK
    return 0;
}

extern "C" int feast_last_profile(double* out)
{
    for (int i = 0; i < 20; ++i) out[i] = g_prof.out[i];
    return 0;
}

// ---------------------------------------------------------------- batched driver
// Many independent problems (FEAST's first level of parallelism: separate
// search intervals) solved together: one filter launch sequence covers the
// work items of every unfinished problem, and the Rayleigh-Ritz step is a
// fixed sequence of batched kernels over all problems.  Both sequences are
// captured once as CUDA graphs (the COCG step index lives on the device) and
// replayed every refinement loop; finished problems are switched off by
// flags in the problem tables.
namespace {

__global__ void kb_col_to_row(const BProb* pr, const double* xc, double* xr)
{
    const BProb& P = pr[blockIdx.y];
    const long long total = (long long)P.n * P.m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / P.m), j = (int)(idx % P.m);
        xr[P.q_off + idx] = xc[P.q_off + (size_t)j * P.n + i];
    }
}

__global__ void kb_random(const BProb* pr, unsigned long long seed, const int* has_x0, double* y)
{
    const BProb& P = pr[blockIdx.y];
    if (has_x0[blockIdx.y]) return;
    const long long total = (long long)P.n * P.m;
    const unsigned long long sd = seed + 0x9E37ull * (unsigned long long)(blockIdx.y + 1);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const unsigned long long h1 = splitmix64(sd * 0x100000001B3ull + 2 * (unsigned long long)idx);
        const unsigned long long h2 = splitmix64(sd * 0x100000001B3ull + 2 * (unsigned long long)idx + 1);
        const double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
        y[P.q_off + idx] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

// column c (column-major, at q_off) = X row-major column perm[l_off + c], 0 beyond mk
__global__ void kb_gather(const BProb* pr, const int* mk, const int* perm, const double* xr, double* xc)
{
    const BProb& P = pr[blockIdx.y];
    const long long total = (long long)P.n * P.m;
    const int k = mk[blockIdx.y];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx / P.n), i = (int)(idx % P.n);
        xc[P.q_off + idx] = c < k ? xr[P.q_off + (size_t)i * P.m + perm[P.l_off + c]] : 0.0;
    }
}

struct Bump {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    T* take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += std::max<size_t>(count, 1) * sizeof(T);
        return p;
    }
};

// rows-per-item choices tried by the autotuner, and the cache of its picks
// keyed by (total rows / 2^16, tile width, precision)
std::vector<std::pair<long long, int>> g_rb_cache;
std::mutex g_rb_mu;

}  // namespace

extern "C" int feast_scsr_solve_batched(int np, const feast_problem* probs, int* fpm, feast_result* out)
{
    if (np <= 0) return -101;
    if (!probs) return -102;
    if (!fpm) return -103;
    if (!out) return -104;
    int inf = check_fpm(fpm);
    if (inf) return inf;
    if (fpm[13] != 0) return 114;  // one-pass modes are single-problem only
    if (fpm[39] != 0) return 140;
    g_err.clear();
    const int ne = fpm[1];
    const bool fp64 = fpm[41] == 0;
    const double eps = std::pow(10.0, -fpm[2]);
    const double tol = std::pow(10.0, -fpm[44]);
    const int maxit = fpm[45], maxloop = fpm[3];
    // ---- host side: validate and expand every CSR
    std::vector<std::vector<int>> aia(np), aja(np), bia(np), bja(np);
    std::vector<std::vector<double>> av(np), bv(np);
    int hasB = -1;
    bool bdiag = true;
    for (int p = 0; p < np; ++p) {
        const feast_problem& q = probs[p];
        out[p].info = 0;
        out[p].m = 0;
        out[p].loop = 0;
        out[p].m0 = q.m0;
        out[p].epsout = 1.0;
        if (q.n <= 0) { out[p].info = 202; return -102; }
        if (q.m0 <= 0 || q.m0 > q.n || q.m0 > 128) { out[p].info = 201; return -102; }
        if (!(q.emin < q.emax)) { out[p].info = 200; return -102; }
        if (!out[p].e || !out[p].x || !out[p].res) return -104;
        int st = host_csr('F', q.n, q.a, q.ia, q.ja, 3, aia[p], aja[p], av[p]);
        if (st) { out[p].info = st; return -102; }
        const int hb = (q.b || q.ib || q.jb) ? 1 : 0;
        if (hasB < 0) hasB = hb;
        if (hasB != hb) return -102;
        if (hb) {
            st = host_csr('F', q.n, q.b, q.ib, q.jb, 6, bia[p], bja[p], bv[p]);
            if (st) { out[p].info = st; return -102; }
            for (int i = 0; i < q.n && bdiag; ++i)
                bdiag = bia[p][i + 1] - bia[p][i] == 1 && bja[p][bia[p][i]] == i;
        }
    }
    const int bmode = hasB ? (bdiag ? 1 : 2) : 0;
    // ---- plan
    int W, nbp, mt;
    const int nb = fpm[49] > 0 ? std::min(fpm[49], ne) : 1;
    feast_filter_layout(nb, fp64 ? 1 : 0, &W, &nbp, &mt);
    const int nbatch = (ne + nbp - 1) / nbp;
    const int RBb = 512;
    const size_t csz = fp64 ? 16 : 8, pkz = fp64 ? 16 : 8;
    std::vector<FiltProb> fpv(np);
    std::vector<BProb> bpv(np);
    std::vector<int> G(np);
    long long rows = 0, vec = 0, qo = 0, dqo = 0, co = 0, gpo = 0, wo = 0, nnzA = 0, nnzB = 0, ppA = 0, pkA = 0,
              ppB = 0, pkB = 0;
    int colo = 0, grpo = 0, lo = 0, gram_b = 0, gemm_b = 0, res_b = 0, maxm = 0;
    for (int p = 0; p < np; ++p) {
        const int n = probs[p].n, m = probs[p].m0;
        G[p] = (m + mt - 1) / mt;
        FiltProb& f = fpv[p];
        memset(&f, 0, sizeof(f));
        f.n = n;
        f.m0 = m;
        f.G = G[p];
        f.nrb_b = (n + RBb - 1) / RBb;
        f.vec_off = vec;
        f.col_off = colo;
        f.grp_off = grpo;
        f.q_off = qo;
        f.dq_off = dqo;
        f.ne = ne;
        f.active = 1;
        BProb& b = bpv[p];
        memset(&b, 0, sizeof(b));
        b.n = n;
        b.m = m;
        b.row0 = rows;
        b.q_off = qo;
        b.c_off = co;
        b.l_off = lo;
        b.gram_T = (m + 63) / 64;
        b.gram_ks = std::max(1, std::min(32, (n + 4095) / 4096));
        b.gram_b0 = gram_b;
        b.gpart_off = gpo;
        b.gemm_b0 = gemm_b;
        b.res_b0 = res_b;
        b.w_off = wo;
        b.alpha = std::max(std::fabs(probs[p].emin), std::fabs(probs[p].emax));
        b.active = 1;
        rows += n;
        vec += (long long)G[p] * n * W;
        colo += G[p] * W;
        grpo += G[p];
        qo += (long long)n * m;
        dqo += (long long)G[p] * n * mt;
        co += (long long)m * m;
        lo += m;
        gram_b += b.gram_T * (b.gram_T + 1) / 2 * b.gram_ks;
        gpo += (long long)b.gram_ks * m * m;
        gemm_b += ((n + 63) / 64) * b.gram_T;
        res_b += (n + 255) / 256;
        wo += 6LL * m * m + 4LL * m;
        nnzA += (long long)aja[p].size();
        nnzB += (long long)bja[p].size();
        ppA += n + 1;
        pkA += (long long)aja[p].size() + 7LL * n;
        if (bmode == 2) {
            ppB += n + 1;
            pkB += (long long)bja[p].size() + 7LL * n;
        }
        maxm = std::max(maxm, m);
    }
    int ga = 1, gb = 1;
    filter_grids(fp64, W, &ga, &gb);
    // partial-sum slots for the smallest row block the tuner may pick
    const int rb_min = fpm[50] > 0 ? std::min(fpm[50], 512) : 128;
    int nslot = 1, nbk = 1;
    for (int p = 0; p < np; ++p) {
        const int nrb_max = (probs[p].n + rb_min - 1) / rb_min;
        nslot = std::max(nslot, std::max(part_slots(nrb_max), part_slots(fpv[p].nrb_b)));
        nbk = std::max(nbk, std::max(part_buckets(nrb_max), part_buckets(fpv[p].nrb_b)));
    }
    // work items of the two COCG steps at the smallest row block (problem lookup tables)
    long long items_a_max = 0, items_b = 0;
    for (int p = 0; p < np; ++p) {
        items_a_max += (long long)G[p] * ((probs[p].n + rb_min - 1) / rb_min);
        items_b += (long long)G[p] * fpv[p].nrb_b;
    }
    // ---- device memory: one allocation carved in place
    DevMem dm;
    Bump bump;
    char* base = nullptr;
    for (int pass = 0; pass < 2; ++pass) {
        bump.base = base;
        bump.off = 0;
        (void)bump.take<int>(ppA);
        (void)bump.take<int>(nnzA);
        (void)bump.take<double>(nnzA);
        (void)bump.take<int>(hasB ? ppA : 0);
        (void)bump.take<int>(nnzB);
        (void)bump.take<double>(nnzB);
        (void)bump.take<int>(ppA);
        (void)bump.take<char>(pkA * pkz);
        (void)bump.take<int>(ppB);
        (void)bump.take<char>(pkB * pkz);
        (void)bump.take<double>(bmode == 1 ? rows : 0);
        (void)bump.take<FiltProb>(np);
        (void)bump.take<BProb>(np);
        (void)bump.take<char>(vec * csz * 3);
        (void)bump.take<ColState>(colo);
        (void)bump.take<double>((size_t)grpo * nslot * W * 4);
        (void)bump.take<unsigned>((size_t)grpo * nbk);
        (void)bump.take<unsigned>(grpo);
        (void)bump.take<int>(grpo);
        (void)bump.take<int>((size_t)nbatch * np);
        (void)bump.take<int>(np);
        (void)bump.take<unsigned long long>(1);
        (void)bump.take<int>(1);
        (void)bump.take<double>((size_t)np * ne * 4);
        (void)bump.take<char>(dqo * (fp64 ? 8 : 4));
        for (int t = 0; t < 6; ++t) (void)bump.take<double>(qo);  // Y, Q, X, T, T2, xc
        for (int t = 0; t < 3; ++t) (void)bump.take<double>(co);  // Aq, Bq, Vr
        (void)bump.take<double>(lo);
        (void)bump.take<double>(lo);
        (void)bump.take<int>(np);
        (void)bump.take<int>(lo);
        (void)bump.take<int>(np);
        (void)bump.take<double>(gpo);
        (void)bump.take<double>((size_t)res_b * 128 * 2);
        (void)bump.take<double>(wo);
        (void)bump.take<int>(items_a_max);
        (void)bump.take<int>(items_b);
        if (pass == 0) {
            cudaError_t e = dm.alloc(&base, bump.off + 4096);
            if (e != cudaSuccess) return cuda_fail(e, "batched workspace");
        }
    }
    bump.base = base;
    bump.off = 0;
    int* d_ia = bump.take<int>(ppA);
    int* d_ja = bump.take<int>(nnzA);
    double* d_a = bump.take<double>(nnzA);
    int* d_ib = bump.take<int>(hasB ? ppA : 0);
    int* d_jb = bump.take<int>(nnzB);
    double* d_b = bump.take<double>(nnzB);
    int* d_app = bump.take<int>(ppA);
    char* d_apk = bump.take<char>(pkA * pkz);
    int* d_bpp = bump.take<int>(ppB);
    char* d_bpk = bump.take<char>(pkB * pkz);
    double* d_bd = bump.take<double>(bmode == 1 ? rows : 0);
    FiltProb* d_fp = bump.take<FiltProb>(np);
    BProb* d_bp = bump.take<BProb>(np);
    char* d_vec = bump.take<char>(vec * csz * 3);
    ColState* d_cs = bump.take<ColState>(colo);
    double* d_part = bump.take<double>((size_t)grpo * nslot * W * 4);
    unsigned* d_bkcount = bump.take<unsigned>((size_t)grpo * nbk);
    unsigned* d_gcount = bump.take<unsigned>(grpo);
    int* d_gdone = bump.take<int>(grpo);
    int* d_itmax = bump.take<int>((size_t)nbatch * np);
    int* d_gleft = bump.take<int>(np);
    unsigned long long* d_work = bump.take<unsigned long long>(1);
    int* d_k = bump.take<int>(1);
    double* d_zw = bump.take<double>((size_t)np * ne * 4);
    char* d_dq = bump.take<char>(dqo * (fp64 ? 8 : 4));
    double* d_Y = bump.take<double>(qo);
    double* d_Q = bump.take<double>(qo);
    double* d_X = bump.take<double>(qo);
    double* d_T = bump.take<double>(qo);
    double* d_T2 = bump.take<double>(qo);
    double* d_xc = bump.take<double>(qo);
    double* d_Aq = bump.take<double>(co);
    double* d_Bq = bump.take<double>(co);
    double* d_Vr = bump.take<double>(co);
    double* d_lam = bump.take<double>(lo);
    double* d_res = bump.take<double>(lo);
    int* d_mk = bump.take<int>(np);
    int* d_perm = bump.take<int>(lo);
    int* d_hasx = bump.take<int>(np);
    double* d_gpart = bump.take<double>(gpo);
    double* d_rpart = bump.take<double>((size_t)res_b * 128 * 2);
    double* d_rwork = bump.take<double>(wo);
    int* d_itp = bump.take<int>(items_a_max);
    int* d_itpb = bump.take<int>(items_b);
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sguard{s};
    // ---- uploads: matrices, packed chunks, tables, nodes, start blocks
    {
        long long oa = 0, onz = 0, ob = 0, onzb = 0, opp = 0, opk = 0, oppb = 0, opkb = 0;
        std::vector<double> zw_all((size_t)np * ne * 4);
        std::vector<int> hasx(np, 0);
        for (int p = 0; p < np; ++p) {
            const int n = probs[p].n;
            CK(cudaMemcpyAsync(d_ia + oa, aia[p].data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(d_ja + onz, aja[p].data(), sizeof(int) * aja[p].size(), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(d_a + onz, av[p].data(), sizeof(double) * av[p].size(), cudaMemcpyHostToDevice, s));
            FiltProb& f = fpv[p];
            BProb& b = bpv[p];
            f.ia = b.ia = d_ia + oa;
            f.ja = b.ja = d_ja + onz;
            f.av = b.av = d_a + onz;
            // padded chunk pointers from the host copy
            std::vector<int> pp(n + 1, 0);
            for (int i = 0; i < n; ++i) pp[i + 1] = pp[i] + (aia[p][i + 1] - aia[p][i] + 7) / 8 * 8;
            CK(cudaMemcpyAsync(d_app + opp, pp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));
            CK(launch_pack_csr(n, d_ia + oa, d_ja + onz, d_a + onz, d_app + opp, fp64, d_apk + opk * pkz, s));
            f.app = d_app + opp;
            f.apk = d_apk + opk * pkz;
            if (hasB) {
                CK(cudaMemcpyAsync(d_ib + ob, bia[p].data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
                CK(cudaMemcpyAsync(d_jb + onzb, bja[p].data(), sizeof(int) * bja[p].size(), cudaMemcpyHostToDevice, s));
                CK(cudaMemcpyAsync(d_b + onzb, bv[p].data(), sizeof(double) * bv[p].size(), cudaMemcpyHostToDevice, s));
                f.ib = b.ib = d_ib + ob;
                f.jb = b.jb = d_jb + onzb;
                f.bv = b.bv = d_b + onzb;
                if (bmode == 1) {
                    CK(launch_cast_diag(n, d_ib + ob, d_b + onzb, fp64, (char*)d_bd + (size_t)b.row0 * (fp64 ? 8 : 4), s));
                    f.bd = (char*)d_bd + (size_t)b.row0 * (fp64 ? 8 : 4);
                } else {
                    std::vector<int> bp(n + 1, 0);
                    for (int i = 0; i < n; ++i) bp[i + 1] = bp[i] + (bia[p][i + 1] - bia[p][i] + 7) / 8 * 8;
                    CK(cudaMemcpyAsync(d_bpp + oppb, bp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
                    CK(cudaStreamSynchronize(s));
                    CK(launch_pack_csr(n, d_ib + ob, d_jb + onzb, d_b + onzb, d_bpp + oppb, fp64, d_bpk + opkb * pkz, s));
                    f.bpp = d_bpp + oppb;
                    f.bpk = d_bpk + opkb * pkz;
                    oppb += n + 1;
                    opkb += (long long)bja[p].size() + 7LL * n;
                }
                ob += n + 1;
                onzb += (long long)bja[p].size();
            }
            oa += n + 1;
            onz += (long long)aja[p].size();
            opp += n + 1;
            opk += (long long)aja[p].size() + 7LL * n;
            std::vector<double> zw;
            contour(fpm[15], ne, probs[p].emin, probs[p].emax, fpm[17] / 100.0, zw);
            std::copy(zw.begin(), zw.end(), zw_all.begin() + (size_t)p * ne * 4);
            f.zw = d_zw + (size_t)p * ne * 4;
            f.lam = d_lam + b.l_off;
            f.mk = d_mk + p;
            if (probs[p].x0) {
                hasx[p] = 1;
                CK(cudaMemcpyAsync(d_xc + b.q_off, probs[p].x0, sizeof(double) * (size_t)n * probs[p].m0,
                                   cudaMemcpyHostToDevice, s));
            }
        }
        CK(cudaMemcpyAsync(d_zw, zw_all.data(), sizeof(double) * zw_all.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_bp, bpv.data(), sizeof(BProb) * np, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_hasx, hasx.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
        std::vector<int> mk0(np);
        for (int p = 0; p < np; ++p) mk0[p] = probs[p].m0;
        CK(cudaMemcpyAsync(d_mk, mk0.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
        // start blocks: given ones transposed to row-major, the others random
        kb_col_to_row<<<dim3(64, np), 256, 0, s>>>(d_bp, d_xc, d_Y);
        const unsigned long long seed = fpm[51] ? (unsigned long long)fpm[51] : 0x5EEDull;
        kb_random<<<dim3(64, np), 256, 0, s>>>(d_bp, seed, d_hasx, d_Y);
        count_launches(2);
        CK(cudaGetLastError());
        // x0 blocks of problems without one are overwritten by the random block
        CK(cudaStreamSynchronize(s));
        for (int p = 0; p < np; ++p)
            if (!probs[p].x0) { /* random block already in d_Y */ }
        CK(cudaMemcpyAsync(d_Q, d_Y, sizeof(double) * qo, cudaMemcpyDeviceToDevice, s));
    }
    // ---- filter tables for a given rows-per-item choice
    long long nitems = 0, nitems_b = 0;
    int RB = 128;
    // problem of every work item (a lookup instead of a binary search of the
    // problem table in every item of every COCG launch)
    std::vector<int> itp, itpb;
    auto build_tables = [&](int rb) -> int {
        RB = rb;
        long long it = 0, itb = 0;
        itp.clear();
        itpb.clear();
        for (int p = 0; p < np; ++p) {
            FiltProb& f = fpv[p];
            f.nrb = (f.n + RB - 1) / RB;
            f.item0 = it;
            f.item0_b = itb;
            it += (long long)f.G * f.nrb;
            itb += (long long)f.G * f.nrb_b;
            itp.insert(itp.end(), (size_t)f.G * f.nrb, p);
            itpb.insert(itpb.end(), (size_t)f.G * f.nrb_b, p);
        }
        nitems = it;
        nitems_b = itb;
        if (it > items_a_max || itb > items_b) return -4;
        CK(cudaMemcpyAsync(d_fp, fpv.data(), sizeof(FiltProb) * np, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_itp, itp.data(), sizeof(int) * itp.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_itpb, itpb.data(), sizeof(int) * itpb.size(), cudaMemcpyHostToDevice, s));
        return 0;
    };
    FilterArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.probs = d_fp;
    fa.nprob = np;
    fa.W = W;
    fa.nbp = nbp;
    fa.mt = mt;
    fa.RBb = RBb;
    fa.hasB = hasB;
    fa.bmode = bmode;
    fa.r = d_vec;
    fa.p0 = d_vec + vec * csz;
    fa.p1 = d_vec + 2 * vec * csz;
    fa.cs = d_cs;
    fa.part = d_part;
    fa.grp_count = d_gcount;
    fa.bk_count = d_bkcount;
    fa.nbk = nbk;
    fa.nslot = nslot;
    fa.grp_done = d_gdone;
    fa.Q = d_Q;
    fa.dQ = d_dq;
    fa.tol2 = tol * tol;
    fa.groups_left = d_gleft;
    fa.work = d_work;
    fa.kdev = d_k;
    fa.iter_max = d_itmax;
    fa.item_prob = d_itp;
    fa.item_prob_b = d_itpb;
    int st = build_tables(fpm[50] > 0 ? std::min(fpm[50], 512) : 256);
    if (st) return st;
    auto grids = [&](int& g_a, int& g_b, int& g_i) {
        g_a = (int)std::min<long long>(ga, std::max(1LL, nitems));
        g_b = (int)std::min<long long>(gb, std::max(1LL, nitems_b));
        g_i = std::max(g_a, g_b);
        fa.nitems = nitems;
        fa.nitems_b = nitems_b;
        fa.RB = RB;
    };
    std::vector<int> gdone(grpo), gleft(np);
    std::vector<char> done(np, 0);
    auto set_groups = [&]() -> int {
        for (int p = 0; p < np; ++p) {
            for (int g = 0; g < G[p]; ++g) gdone[fpv[p].grp_off + g] = done[p] ? 1 : 0;
            gleft[p] = done[p] ? 0 : G[p];
        }
        CK(cudaMemcpyAsync(d_gdone, gdone.data(), sizeof(int) * grpo, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_gleft, gleft.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
        return 0;
    };
    // ---- COCG chunk graph: (step A, step B, k += 1) x 8, step index on the device
    cudaGraphExec_t chunk_exec = nullptr, rr_exec = nullptr;
    struct GraphGuard {
        cudaGraphExec_t* a;
        cudaGraphExec_t* b;
        ~GraphGuard()
        {
            if (*a) cudaGraphExecDestroy(*a);
            if (*b) cudaGraphExecDestroy(*b);
        }
    } gguard{&chunk_exec, &rr_exec};
    auto capture_chunk = [&]() -> int {
        if (chunk_exec) {
            cudaGraphExecDestroy(chunk_exec);
            chunk_exec = nullptr;
        }
        int g_a, g_b, g_i;
        grids(g_a, g_b, g_i);
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int t = 0; t < 8; ++t) {
            launch_cocg_step_a(fa, fp64, 0, g_a, s);
            launch_cocg_step_b(fa, fp64, 0, g_b, s);
            launch_advance(d_k, s);
        }
        CK(cudaStreamEndCapture(s, &graph));
        cudaError_t e = cudaGraphInstantiate(&chunk_exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        return 0;
    };
    // ---- autotuner: time step A (first step, no state change) for a few
    // rows-per-item choices on this batch, keep the fastest
    if (fpm[50] == 0) {
        const long long key = (rows >> 16) * 64 + W * 2 + (fp64 ? 1 : 0);
        int cached = 0;
        {
            std::lock_guard<std::mutex> lock(g_rb_mu);
            for (auto& kv : g_rb_cache)
                if (kv.first == key) cached = kv.second;
        }
        if (!cached) {
            { const int sg = set_groups(); if (sg) return sg; }
            CK(cudaMemsetAsync(d_gcount, 0, sizeof(unsigned) * grpo, s));
            CK(cudaMemsetAsync(d_bkcount, 0, sizeof(unsigned) * (size_t)grpo * nbk, s));
            CK(launch_colstate_init(fa, 0, 0, s));
            float best = 1e30f;
            int best_rb = 256;
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            for (int cand : {128, 256, 512}) {
                { const int bt = build_tables(cand); if (bt) return bt; }
                int g_a, g_b, g_i;
                grids(g_a, g_b, g_i);
                fa.kdev = nullptr;
                CK(launch_filter_init(fa, fp64, d_Y, d_X, 0, 1, g_i, s));
                CK(launch_cocg_step_a(fa, fp64, 0, g_a, s));
                CK(cudaEventRecord(e0, s));
                for (int t = 0; t < 2; ++t) CK(launch_cocg_step_a(fa, fp64, 0, g_a, s));
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; best_rb = cand; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            fa.kdev = d_k;
            cached = best_rb;
            std::lock_guard<std::mutex> lock(g_rb_mu);
            g_rb_cache.push_back({key, best_rb});
        }
        { const int bt = build_tables(cached); if (bt) return bt; }
        // the timing runs reset Q: start again from the start blocks
        CK(cudaMemcpyAsync(d_Q, d_Y, sizeof(double) * qo, cudaMemcpyDeviceToDevice, s));
    }
    st = capture_chunk();
    if (st) return st;
    // ---- Rayleigh-Ritz graph
    {
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        launch_b_spmm(d_bp, np, rows, d_Q, d_T, 0, s);
        launch_b_gram(d_bp, np, gram_b, maxm, d_Q, d_T, d_gpart, d_Aq, s);
        if (hasB) {
            launch_b_spmm(d_bp, np, rows, d_Q, d_T2, 1, s);
            launch_b_gram(d_bp, np, gram_b, maxm, d_Q, d_T2, d_gpart, d_Bq, s);
        } else {
            launch_b_gram(d_bp, np, gram_b, maxm, d_Q, d_Q, d_gpart, d_Bq, s);
        }
        launch_b_reduced(d_bp, np, d_Aq, d_Bq, d_lam, d_Vr, d_mk, d_rwork, s);
        launch_b_gemm(d_bp, np, gemm_b, d_Q, d_Vr, d_X, s);
        launch_b_residual(d_bp, np, res_b, d_X, d_lam, d_Y, d_rpart, d_res, s);
        CK(cudaStreamEndCapture(s, &graph));
        cudaError_t e = cudaGraphInstantiate(&rr_exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
    }
    // ---- refinement loops
    std::vector<double> lam(lo), res(lo), trace_prev(np, 0.0);
    std::vector<int> mk(np), maxres_ok(np, 0);
    long long total_steps = 0;
    int k = 0;
    for (k = 0;; ++k) {
        CK(cudaGraphLaunch(rr_exec, s));
        CK(cudaMemcpyAsync(lam.data(), d_lam, sizeof(double) * lo, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(res.data(), d_res, sizeof(double) * lo, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(mk.data(), d_mk, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        int left = 0;
        for (int p = 0; p < np; ++p) {
            if (done[p]) continue;
            const BProb& b = bpv[p];
            const double* L = lam.data() + b.l_off;
            const double* Rr = res.data() + b.l_off;
            const double emin = probs[p].emin, emax = probs[p].emax;
            int M = 0;
            double tr = 0.0, mr = 0.0;
            for (int j = 0; j < mk[p]; ++j)
                if (L[j] >= emin && L[j] <= emax) {
                    ++M;
                    tr += L[j];
                    mr = std::max(mr, Rr[j]);
                }
            const double eo = k == 0 ? 1.0 : std::fabs(tr - trace_prev[p]) / b.alpha;
            trace_prev[p] = tr;
            out[p].m = M;
            out[p].loop = k;
            out[p].epsout = eo;
            out[p].m0 = mk[p];
            int info = -1;
            if (mk[p] < 1) info = -3;
            else if (M >= 1 && (fpm[5] == 1 ? mr < eps : (k >= 1 && eo < eps))) info = M >= mk[p] ? 3 : 0;
            else if (M == 0 && k >= 1) info = 1;
            else if (k >= maxloop) info = 2;
            if (info != -1) {
                out[p].info = info;
                done[p] = 1;
                bpv[p].active = 0;
                fpv[p].active = 0;
            } else {
                ++left;
            }
        }
        CK(cudaMemcpyAsync(d_bp, bpv.data(), sizeof(BProb) * np, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_fp, fpv.data(), sizeof(FiltProb) * np, cudaMemcpyHostToDevice, s));
        if (!left) break;
        // residual-inverse filter pass over the unfinished problems
        { const int sg = set_groups(); if (sg) return sg; }
        int g_a, g_b, g_i;
        grids(g_a, g_b, g_i);
        for (int bt = 0; bt < nbatch; ++bt) {
            CK(cudaMemsetAsync(d_gcount, 0, sizeof(unsigned) * grpo, s));
            CK(cudaMemsetAsync(d_bkcount, 0, sizeof(unsigned) * (size_t)grpo * nbk, s));
            { const int sg = set_groups(); if (sg) return sg; }
            CK(cudaMemsetAsync(d_k, 0, sizeof(int), s));
            CK(launch_colstate_init(fa, bt * nbp, 1, s));
            CK(launch_filter_init(fa, fp64, d_Y, d_X, 1, bt == 0, g_i, s));
            for (int c = 0; c * 8 < maxit; ++c) {
                CK(cudaGraphLaunch(chunk_exec, s));
                total_steps += 8;
                CK(cudaMemcpyAsync(gleft.data(), d_gleft, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                int any = 0;
                for (int p = 0; p < np; ++p) any += gleft[p] > 0;
                if (!any) break;
            }
        }
        CK(launch_fold_dq(fa, qo, fp64, s));
    }
    fpm[59] = (int)std::min<long long>(total_steps, 2147483647LL);
    // ---- outputs: inside ascending, then outside ascending
    std::vector<int> perm(lo, 0);
    for (int p = 0; p < np; ++p) {
        const BProb& b = bpv[p];
        const double* L = lam.data() + b.l_off;
        const double* Rr = res.data() + b.l_off;
        int c = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < mk[p]; ++j) {
                const bool in = L[j] >= probs[p].emin && L[j] <= probs[p].emax;
                if ((pass == 0) == in) perm[b.l_off + c++] = j;
            }
        for (int j = 0; j < probs[p].m0; ++j) {
            out[p].e[j] = j < mk[p] ? L[perm[b.l_off + j]] : 0.0;
            out[p].res[j] = j < mk[p] ? Rr[perm[b.l_off + j]] : 0.0;
        }
    }
    CK(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * lo, cudaMemcpyHostToDevice, s));
    kb_gather<<<dim3(64, np), 256, 0, s>>>(d_bp, d_mk, d_perm, d_X, d_xc);
    count_launches(1);
    CK(cudaGetLastError());
    for (int p = 0; p < np; ++p)
        CK(cudaMemcpyAsync(out[p].x, d_xc + bpv[p].q_off, sizeof(double) * (size_t)probs[p].n * probs[p].m0,
                           cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    (void)k;
    return 0;
}

// ---------------------------------------------------------------- helpers for the Hermitian driver
namespace feast {
int fpm_check(const int* fpm) { return check_fpm(fpm); }
void contour_nodes(int rule, int ne, double emin, double emax, double ratio, std::vector<double>& zw)
{
    contour(rule, ne, emin, emax, ratio, zw);
}
int cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }
void clear_last_error() { g_err.clear(); }
void feast_log(int lvl, const char* text) { log_line(lvl, text); }
}  // namespace feast
