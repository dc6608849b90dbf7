// Complex Hermitian FEAST kernels (FEAST v4.0 guide, Sec. 3.2 "FEAST
// Hermitian", zfeast_hcsr{ev,gv}): A Hermitian, B Hermitian positive definite,
// both as CSR with complex double values.
//
// Filter.  With G(z) = (zB - A)^{-1} the lower half contour is no longer the
// conjugate of the upper one, so each node z_e needs G(z_e) and G(conj z_e):
//   Q = sum_e (1/2)[w_e G(z_e) + conj(w_e) G(conj z_e)] B Y          (first pass)
//   Q = X rho(Lambda) + sum_e (1/2)[c_e y_e + conj(c_e) yh_e]       (residual-inverse passes)
// with c_e = w_e / (z_e - lambda_j), y_e = G(z_e) r_j, yh_e = G(conj z_e) r_j.
// K = z_e B - A has K^H = conj(z_e) B - A, so one BiCG run on K with the
// shadow system K^H and the shadow right-hand side equal to the primal one
// yields both solutions; the shadow system uses the same A and B entries with
// the conjugate shift.  For real A, B and b this is COCG (the shadow iterates
// are the conjugates of the primal ones).  The solutions are never stored:
// every step adds (1/2)(c alpha p + conj(c alpha) ph) to the quadrature block.
//
// Lanes and layout.  A lane is one (node, column) pair; block vectors are
// row-major n x L complex (L = nodes x columns, node fastest), so the lanes of
// one row are one contiguous segment and a warp covers 32 lanes of a row.
// One BiCG step is four launches:
//   step_a    s = K r, sh = K^H rh (one pass over the row entries for both),
//             p = r + beta p, ph = rh + conj(beta) ph, q = s + beta q,
//             qh = sh + conj(beta) qh, per-row-block partials of ph^H q
//   finish_a  alpha = rho / (ph^H q) per lane (fixed-order sum of partials)
//   step_b    r -= alpha q, rh -= conj(alpha) qh, dQ += (1/2)(c alpha p +
//             conj(c alpha) ph) summed over the node lanes of a column, and
//             partials of rh^H r, |r|^2, |rh|^2
//   finish_b  beta = rho_new / rho, convergence (|r|, |rh| <= tol |b|) and
//             breakdown per lane
// Reductions are deterministic: per row block fixed-order partial sums, then a
// fixed-order sum over the row blocks.
#include <algorithm>

#include "feast_internal.cuh"
#include "herm_internal.cuh"

namespace feast {
namespace herm {

static constexpr int kT = 256;   // threads per CTA

template <typename V> __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cadd2(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
// conj(a) * b
template <typename V> __device__ __forceinline__ V cmulc(V a, V b)
{
    return cmk<V>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
template <typename V> __device__ __forceinline__ V from_d2(double2 v);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }

// y = sum_k a_k x[j_k], yh = sum_k a_k xh[j_k] over the CSR row (complex values
// a, complex x with row stride L), four entries at a time: their column indices
// first, then all eight gathers, so they are in flight together.
template <typename T>
__device__ __forceinline__ void row_pair(const int* __restrict__ ia, const int* __restrict__ ja,
                                         const c2_t<T>* __restrict__ av, int i, const c2_t<T>* __restrict__ x,
                                         const c2_t<T>* __restrict__ xh, long long L, c2_t<T>& y, c2_t<T>& yh)
{
    using V = c2_t<T>;
    constexpr int U = 4;
    y = cmk<V>(T(0), T(0));
    yh = y;
    const int s = __ldg(ia + i), e = __ldg(ia + i + 1);
    for (int k = s; k < e; k += U) {
        long long j[U];
        V a[U], xv[U], xhv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = k + u < e;
            j[u] = ok ? __ldg(ja + k + u) : -1;
            a[u] = ok ? av[k + u] : cmk<V>(T(0), T(0));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xv[u] = j[u] >= 0 ? __ldg(x + j[u] * L) : cmk<V>(T(0), T(0));
            xhv[u] = j[u] >= 0 ? __ldg(xh + j[u] * L) : cmk<V>(T(0), T(0));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            y = cfma(a[u], xv[u], y);
            yh = cfma(a[u], xhv[u], yh);
        }
    }
}

// ---------------------------------------------------------------- lanes and setup
// Lanes per column: the node count of the batch rounded up to a power of two,
// so a column's node lanes are an aligned group inside one warp and are
// summed by shuffles.  Padding lanes never iterate.
__host__ __device__ inline int lanes_per_col(int nb)
{
    int p = 1;
    while (p < nb) p <<= 1;
    return p;
}

// rho(l) = sum_e Re(w_e / (z_e - l)) over all nodes of the contour.
__device__ double rho_of(const double* zw, int ne, double l)
{
    double s = 0.0;
    for (int e = 0; e < ne; ++e) {
        const double zr = zw[4 * e] - l, zi = zw[4 * e + 1], wr = zw[4 * e + 2], wi = zw[4 * e + 3];
        s += (wr * zr + wi * zi) / (zr * zr + zi * zi);
    }
    return s;
}

// Lane state.  zwb: the batch's nodes [nb][4]; lam: Ritz values (rii).
__global__ void h_lane_init(HArgs a, const double* __restrict__ zwb, const double* __restrict__ lam, int rii)
{
    const int nbp = lanes_per_col(a.nb);
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < a.L; l += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(l % nbp), j = (int)(l / nbp);
        HLane s;
        s.rho = s.alpha = s.beta = s.z = s.c = make_double2(0.0, 0.0);
        s.bn2 = s.rn2 = s.rhn2 = 0.0;
        s.iters = 0;
        s.active = e < a.nb && j < a.m;
        s.status = s.active ? 0 : 3;
        if (s.active) {
            const double zr = zwb[4 * e], zi = zwb[4 * e + 1], wr = zwb[4 * e + 2], wi = zwb[4 * e + 3];
            s.z = make_double2(zr, zi);
            if (rii) {  // c = w / (z - lambda_j)
                const double dr = zr - lam[j], den = dr * dr + zi * zi;
                s.c = make_double2((wr * dr + wi * zi) / den, (wi * dr - wr * zi) / den);
            } else {
                s.c = make_double2(wr, wi);
            }
        }
        a.st[l] = s;
    }
}

// r = rh = b (b: n x m FP64, row-major) for every lane of column j; with
// init_q the quadrature block starts at X rho(lam) (rii) or zero.
template <typename T>
__global__ void __launch_bounds__(kT) h_vec_init(HArgs a, const double2* __restrict__ b, const double2* __restrict__ X,
                                                 const double* __restrict__ lam, const double* __restrict__ zw_all,
                                                 int ne_all, int rii, int init_q)
{
    using V = c2_t<T>;
    const int nbp = lanes_per_col(a.nb);
    V* r = (V*)a.r;
    V* rh = (V*)a.rh;
    const long long total = (long long)a.n * a.L;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / a.L, l = idx % a.L;
        const int e = (int)(l % nbp), j = (int)(l / nbp);
        V v = cmk<V>(T(0), T(0));
        if (e < a.nb && j < a.m) v = from_d2<V>(b[i * a.m + j]);
        r[idx] = v;
        rh[idx] = v;
        if (init_q && e == 0 && j < a.m) {
            double2 qv = make_double2(0.0, 0.0);
            if (rii) {
                const double f = rho_of(zw_all, ne_all, lam[j]);
                const double2 x = X[i * a.m + j];
                qv = make_double2(f * x.x, f * x.y);
            }
            a.Q[i * a.m + j] = qv;
            if (a.dQ) ((float2*)a.dQ)[i * a.m + j] = make_float2(0.f, 0.f);
        }
    }
}

// ---------------------------------------------------------------- BiCG steps
// Work item = (row block of kRowsPerItem rows, chunk of 32 lanes); warp w of
// the CTA takes rows w, w + 8, ... of the block, one lane per thread.  The
// per-lane partial sums of the item (fixed order over its warps) go to
// part[rb][v][l].
__device__ __forceinline__ void item_sum(double2 v, double2 (*sh)[32], double2* __restrict__ out, bool ok)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    sh[warp][lane] = v;
    __syncthreads();
    if (warp == 0 && ok) {
        double2 s = sh[0][lane];
        for (int w = 1; w < kT / 32; ++w) {
            s.x += sh[w][lane].x;
            s.y += sh[w][lane].y;
        }
        *out = s;
    }
    __syncthreads();
}

// partials of |r|^2 (setup of |b|^2)
template <typename T>
__global__ void __launch_bounds__(kT) h_norms(HArgs a)
{
    using V = c2_t<T>;
    __shared__ double2 sh[kT / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nrbk = row_blocks(a.n);
    const long long nch = (a.L + 31) / 32, items = (long long)nrbk * nch;
    const V* r = (const V*)a.r;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int rb = (int)(it % nrbk);  // lane chunk major: concurrent items sweep one chunk's rows
        const long long l = (it / nrbk) * 32 + lane;
        const bool ok = l < a.L;
        T acc = T(0);  // per-thread partial in the filter precision (GB300's FP64 ALU is slow)
        if (ok && a.st[l].active) {
            const int i1 = min(a.n, (rb + 1) * kRowsPerItem);
            for (int i = rb * kRowsPerItem + warp; i < i1; i += kT / 32) {
                const V v = r[(long long)i * a.L + l];
                acc = fma(v.x, v.x, fma(v.y, v.y, acc));
            }
        }
        item_sum(make_double2((double)acc, 0.0), sh, a.part + ((long long)rb * 2) * a.L + l, ok);
    }
}

template <typename T>
__global__ void __launch_bounds__(kT) h_step_a(HArgs a)
{
    using V = c2_t<T>;
    __shared__ double2 sh[kT / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nrbk = row_blocks(a.n);
    const long long nch = (a.L + 31) / 32, items = (long long)nrbk * nch;
    const long long L = a.L;
    const V* r = (const V*)a.r;
    const V* rh = (const V*)a.rh;
    V* p = (V*)a.p;
    V* ph = (V*)a.ph;
    V* q = (V*)a.q;
    V* qh = (V*)a.qh;
    const V* av = (const V*)a.av;
    const V* bv = (const V*)a.bv;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int rb = (int)(it % nrbk);  // lane chunk major: concurrent items sweep one chunk's rows
        const long long l = (it / nrbk) * 32 + lane;
        const bool ok = l < L;
        V acc = cmk<V>(T(0), T(0));  // per-thread partial of ph^H q, filter precision
        if (ok && a.st[l].active) {
            const HLane& s = a.st[l];
            const bool first = s.iters == 0;
            const V z = from_d2<V>(s.z), zc = cconj(z);
            const V bt = from_d2<V>(s.beta), btc = cconj(bt);
            const int i1 = min(a.n, (rb + 1) * kRowsPerItem);
            for (int i = rb * kRowsPerItem + warp; i < i1; i += kT / 32) {
                const long long o = (long long)i * L + l;
                V ar, arh, br, brh;
                row_pair<T>(a.ia, a.ja, av, i, r + l, rh + l, L, ar, arh);
                if (a.ib) {
                    row_pair<T>(a.ib, a.jb, bv, i, r + l, rh + l, L, br, brh);
                } else {
                    br = r[o];
                    brh = rh[o];
                }
                const V sv = csub(cmul(z, br), ar);     // (z B - A) r
                const V shv = csub(cmul(zc, brh), arh);  // (conj z B - A) rh
                V pn, phn, qn, qhn;
                if (first) {
                    pn = r[o];
                    phn = rh[o];
                    qn = sv;
                    qhn = shv;
                } else {
                    pn = cfma(bt, p[o], r[o]);
                    phn = cfma(btc, ph[o], rh[o]);
                    qn = cfma(bt, q[o], sv);
                    qhn = cfma(btc, qh[o], shv);
                }
                p[o] = pn;
                ph[o] = phn;
                q[o] = qn;
                qh[o] = qhn;
                const V u = cmulc(phn, qn);  // conj(ph) q
                acc.x += u.x;
                acc.y += u.y;
            }
        }
        item_sum(to_d2(acc), sh, a.part + ((long long)rb * 2) * L + l, ok);
    }
}

template <typename T>
__global__ void __launch_bounds__(kT) h_step_b(HArgs a)
{
    using V = c2_t<T>;
    __shared__ double2 sh[kT / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nbp = lanes_per_col(a.nb);
    const int nrbk = row_blocks(a.n);
    const long long nch = (a.L + 31) / 32, items = (long long)nrbk * nch;
    const long long L = a.L;
    V* r = (V*)a.r;
    V* rh = (V*)a.rh;
    const V* p = (const V*)a.p;
    const V* ph = (const V*)a.ph;
    const V* q = (const V*)a.q;
    const V* qh = (const V*)a.qh;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int rb = (int)(it % nrbk);  // lane chunk major: concurrent items sweep one chunk's rows
        const long long l = (it / nrbk) * 32 + lane;
        const bool ok = l < L;
        const bool act = ok && a.st[l].active;
        const int e = (int)(l % nbp), j = (int)(l / nbp);
        // any lane of this column still iterating (the column's lanes are an
        // aligned group of nbp lanes of this warp)
        unsigned any = act ? 1u : 0u;
        for (int off = 1; off < nbp; off <<= 1) any |= __shfl_xor_sync(0xffffffffu, any, off);
        V al = cmk<V>(T(0), T(0)), ca = al;
        if (act) {
            const double2 alpha = a.st[l].alpha, c = a.st[l].c;
            al = from_d2<V>(alpha);
            ca = from_d2<V>(make_double2(c.x * alpha.x - c.y * alpha.y, c.x * alpha.y + c.y * alpha.x));
        }
        const V alc = cconj(al);
        // per-thread partials in the filter precision (GB300's FP64 ALU is slow);
        // the item sums and the quadrature block stay FP64
        V rho = cmk<V>(T(0), T(0));
        T nr0 = T(0), nr1 = T(0);
        const int i1 = min(a.n, (rb + 1) * kRowsPerItem);
        // mixed precision: the pass's quadrature sum accumulates in complex FP32
        // (dQ, folded into Q once per pass); FP64 solves add to Q directly
        float2* const dq = (float2*)a.dQ;
        for (int i = rb * kRowsPerItem + warp; i < i1; i += kT / 32) {  // bounds uniform over the warp
            const long long o = (long long)i * L + l;
            const long long qi = (long long)i * a.m + j;
            const bool writes = ok && any && e == 0 && j < a.m;
            double2 qold = make_double2(0.0, 0.0);
            float2 dold = make_float2(0.f, 0.f);
            if (writes) {  // issued with the vector loads
                if (dq) dold = dq[qi];
                else qold = a.Q[qi];
            }
            V d = cmk<V>(T(0), T(0));
            if (act) {
                const V rn = cfma(cmk<V>(-al.x, -al.y), q[o], r[o]);
                const V rhn = cfma(cmk<V>(-alc.x, -alc.y), qh[o], rh[o]);
                r[o] = rn;
                rh[o] = rhn;
                const V u = cmulc(rhn, rn);
                rho.x += u.x;
                rho.y += u.y;
                nr0 = fma(rn.x, rn.x, fma(rn.y, rn.y, nr0));
                nr1 = fma(rhn.x, rhn.x, fma(rhn.y, rhn.y, nr1));
                // (1/2)(c alpha p + conj(c alpha) ph)
                const V pd = p[o], phd = ph[o];
                d.x = T(0.5) * ((ca.x * pd.x - ca.y * pd.y) + (ca.x * phd.x + ca.y * phd.y));
                d.y = T(0.5) * ((ca.x * pd.y + ca.y * pd.x) + (ca.x * phd.y - ca.y * phd.x));
            }
            for (int off = 1; off < nbp; off <<= 1) {
                d.x += __shfl_xor_sync(0xffffffffu, d.x, off);
                d.y += __shfl_xor_sync(0xffffffffu, d.y, off);
            }
            if (writes) {
                if (dq) dq[qi] = make_float2(dold.x + (float)d.x, dold.y + (float)d.y);
                else a.Q[qi] = make_double2(qold.x + (double)d.x, qold.y + (double)d.y);
            }
        }
        item_sum(to_d2(rho), sh, a.part + ((long long)rb * 2) * L + l, ok);
        item_sum(make_double2((double)nr0, (double)nr1), sh, a.part + ((long long)rb * 2 + 1) * L + l, ok);
    }
}

// ---------------------------------------------------------------- per-lane finish
// Fixed-order sum over the row blocks of part[rb][v][l]: CTA per 32 lanes,
// warp w takes row blocks w, w + 8, ...; then the warps in order.
__device__ __forceinline__ double2 lane_total(const double2* __restrict__ part, int nrbk, long long L, int v,
                                              long long l, double2 (*sh)[32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double2 s = make_double2(0.0, 0.0);
    if (l < L)
        for (int rb = warp; rb < nrbk; rb += kT / 32) {
            const double2 u = part[((long long)rb * 2 + v) * L + l];
            s.x += u.x;
            s.y += u.y;
        }
    sh[warp][lane] = s;
    __syncthreads();
    double2 t = sh[0][lane];
    for (int w = 1; w < kT / 32; ++w) {
        t.x += sh[w][lane].x;
        t.y += sh[w][lane].y;
    }
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kT) h_finish_norms(HArgs a)
{
    __shared__ double2 sh[kT / 32][32];
    const long long l = blockIdx.x * 32LL + (threadIdx.x & 31);
    const double2 t = lane_total(a.part, row_blocks(a.n), a.L, 0, l, sh);
    if (threadIdx.x < 32 && l < a.L && a.st[l].active) {
        HLane& s = a.st[l];
        s.bn2 = s.rn2 = s.rhn2 = t.x;
        s.rho = make_double2(t.x, 0.0);
        if (!(t.x > 0.0)) {  // zero right-hand side: the solution is zero
            s.active = 0;
            s.status = 1;
        }
    }
}

__global__ void __launch_bounds__(kT) h_finish_a(HArgs a)
{
    __shared__ double2 sh[kT / 32][32];
    const long long l = blockIdx.x * 32LL + (threadIdx.x & 31);
    const double2 sg = lane_total(a.part, row_blocks(a.n), a.L, 0, l, sh);
    if (threadIdx.x < 32 && l < a.L && a.st[l].active) {
        HLane& s = a.st[l];
        const double den = sg.x * sg.x + sg.y * sg.y;
        if (!(den > 0.0) || !isfinite(den)) {  // ph^H K p = 0: breakdown
            s.active = 0;
            s.status = 2;
            s.alpha = make_double2(0.0, 0.0);
        } else {  // alpha = rho / sigma
            s.alpha = make_double2((s.rho.x * sg.x + s.rho.y * sg.y) / den, (s.rho.y * sg.x - s.rho.x * sg.y) / den);
        }
    }
}

__global__ void __launch_bounds__(kT) h_finish_b(HArgs a, int maxit)
{
    __shared__ double2 sh[kT / 32][32];
    const long long l = blockIdx.x * 32LL + (threadIdx.x & 31);
    const int nrbk = row_blocks(a.n);
    const double2 rn = lane_total(a.part, nrbk, a.L, 0, l, sh);
    const double2 nr = lane_total(a.part, nrbk, a.L, 1, l, sh);
    if (threadIdx.x < 32 && l < a.L && a.st[l].active) {
        HLane& s = a.st[l];
        s.iters += 1;
        s.rn2 = nr.x;
        s.rhn2 = nr.y;
        const double den = s.rho.x * s.rho.x + s.rho.y * s.rho.y;
        if (nr.x <= a.tol2 * s.bn2 && nr.y <= a.tol2 * s.bn2) {
            s.active = 0;
            s.status = 1;
        } else if (!isfinite(nr.x) || !isfinite(nr.y) || !(rn.x * rn.x + rn.y * rn.y > 0.0) || !(den > 0.0)) {
            s.active = 0;
            s.status = 2;
        } else if (s.iters >= maxit) {  // stopped with an inexact solve
            s.active = 0;
            s.status = 4;
            atomicAdd(a.nactive + 1, 1);
        } else {  // beta = rho_new / rho
            s.beta = make_double2((rn.x * s.rho.x + rn.y * s.rho.y) / den, (rn.y * s.rho.x - rn.x * s.rho.y) / den);
            s.rho = rn;
        }
        if (s.active) atomicAdd(a.nactive, 1);
    }
}

__global__ void h_fold(long long total, const float2* __restrict__ dQ, double2* __restrict__ Q)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const float2 d = dQ[t];
        double2 q = Q[t];
        q.x += (double)d.x;
        q.y += (double)d.y;
        Q[t] = q;
    }
}

// ---------------------------------------------------------------- filter launchers
static int item_grid(const HArgs& a)
{
    const long long items = (long long)row_blocks(a.n) * ((a.L + 31) / 32);
    const long long cap = (long long)num_sms() * (2048 / kT);
    return (int)(items < cap ? (items > 0 ? items : 1) : cap);
}
static int lane_grid(const HArgs& a) { return (int)((a.L + 31) / 32); }

cudaError_t launch_h_init(const HArgs& a, bool fp64, const double2* b, const double2* X, const double* zwb,
                          const double* lam, int rii, int ne_all, const double* zw_all, int init_q, cudaStream_t s)
{
    if (a.n <= 0 || a.L <= 0) return cudaSuccess;
    h_lane_init<<<(int)((a.L + 255) / 256), 256, 0, s>>>(a, zwb, lam, rii);
    const long long total = (long long)a.n * a.L;
    long long blocks = (total + kT - 1) / kT;
    const long long cap = (long long)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (fp64) h_vec_init<double><<<(int)blocks, kT, 0, s>>>(a, b, X, lam, zw_all, ne_all, rii, init_q);
    else h_vec_init<float><<<(int)blocks, kT, 0, s>>>(a, b, X, lam, zw_all, ne_all, rii, init_q);
    if (fp64) h_norms<double><<<item_grid(a), kT, 0, s>>>(a);
    else h_norms<float><<<item_grid(a), kT, 0, s>>>(a);
    h_finish_norms<<<lane_grid(a), kT, 0, s>>>(a);
    count_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_h_fold(const HArgs& a, cudaStream_t s)
{
    const long long total = (long long)a.n * a.m;
    if (!a.dQ || total <= 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    h_fold<<<(int)blocks, 256, 0, s>>>(total, (const float2*)a.dQ, a.Q);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_h_step(const HArgs& a, bool fp64, int maxit, cudaStream_t s)
{
    if (a.n <= 0 || a.L <= 0) return cudaSuccess;
    const int g = item_grid(a), gl = lane_grid(a);
    if (fp64) h_step_a<double><<<g, kT, 0, s>>>(a);
    else h_step_a<float><<<g, kT, 0, s>>>(a);
    h_finish_a<<<gl, kT, 0, s>>>(a);
    if (fp64) h_step_b<double><<<g, kT, 0, s>>>(a);
    else h_step_b<float><<<g, kT, 0, s>>>(a);
    cudaError_t e = cudaMemsetAsync(a.nactive, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    h_finish_b<<<gl, kT, 0, s>>>(a, maxit);
    count_launches(4);
    return cudaGetLastError();
}

__global__ void h_cast_kernel(const double2* __restrict__ src, float2* __restrict__ dst, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

cudaError_t launch_h_cast(const double2* src, void* dst, long long n, bool fp64, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (fp64) return cudaMemcpyAsync(dst, src, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s);
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    h_cast_kernel<<<(int)blocks, 256, 0, s>>>(src, (float2*)dst, n);
    count_launches(1);
    return cudaGetLastError();
}

// ================================================================ Rayleigh-Ritz (FP64 complex)
// Y = A X for row-major n x m complex blocks: warp per row, lanes over columns.
__global__ void __launch_bounds__(256) h_spmm(int n, int m, const int* __restrict__ ia, const int* __restrict__ ja,
                                              const double2* __restrict__ av, const double2* __restrict__ X,
                                              double2* __restrict__ Y)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nwarps) {
        const int s = __ldg(ia + i), e = __ldg(ia + i + 1);
        for (int c = lane; c < m; c += 32) {
            double2 acc = make_double2(0.0, 0.0);
            for (int k = s; k < e; ++k) {
                const double2 a = av[k], x = X[(long long)__ldg(ja + k) * m + c];
                acc.x = fma(a.x, x.x, fma(-a.y, x.y, acc.x));
                acc.y = fma(a.x, x.y, fma(a.y, x.x, acc.y));
            }
            Y[(long long)i * m + c] = acc;
        }
    }
}

cudaError_t launch_h_spmm(int n, int m, const int* ia, const int* ja, const double2* av, const double2* X, double2* Y,
                          cudaStream_t s)
{
    if (n <= 0 || m <= 0) return cudaSuccess;
    long long blocks = ((long long)n + 7) / 8;
    const long long cap = (long long)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    h_spmm<<<(int)blocks, 256, 0, s>>>(n, m, ia, ja, av, X, Y);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- complex FP64 tensor-core tile
// 64 x 64 complex output tile per CTA of 128 threads (2 x 2 warps of 32 x 32),
// K staged 16 at a time in K-major shared tiles (leading dimension 68).
// With the operands split into real and imaginary planes,
//   Re C += Ar Br - Ai Bi,  Im C += Ar Bi + Ai Br,
// four m8n8k4 FP64 MMAs per fragment pair.
static constexpr int HM = 64, HK = 16, HLD = HM + 4;

__device__ __forceinline__ void hmma(double& c0, double& c1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

struct HTiles {
    double ar[HK][HLD], ai[HK][HLD], br[HK][HLD], bi[HK][HLD];
};

__device__ __forceinline__ void htile_mma(const HTiles& t, double (&re)[4][4][2], double (&im)[4][4][2], int wr, int wc,
                                          int lane)
{
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int kk = 0; kk < HK; kk += 4) {
        double xr[4], xi[4], yr[4], yi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xr[i] = t.ar[kk + q][wr + i * 8 + g];
            xi[i] = t.ai[kk + q][wr + i * 8 + g];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            yr[j] = t.br[kk + q][wc + j * 8 + g];
            yi[j] = t.bi[kk + q][wc + j * 8 + g];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                hmma(re[i][j][0], re[i][j][1], xr[i], yr[j]);
                hmma(re[i][j][0], re[i][j][1], -xi[i], yi[j]);
                hmma(im[i][j][0], im[i][j][1], xr[i], yi[j]);
                hmma(im[i][j][0], im[i][j][1], xi[i], yr[j]);
            }
    }
}

__device__ __forceinline__ void hzero(double (&v)[4][4][2])
{
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) v[i][j][0] = v[i][j][1] = 0.0;
}

// Store the warp's 32 x 32 fragment of (re, im) to out (row-major, leading
// dimension ld, rows < nr, cols < nc), tile origin (r0, c0).
__device__ __forceinline__ void hstore(const double (&re)[4][4][2], const double (&im)[4][4][2], double2* out,
                                       long long ld, int nr, int nc, int r0, int c0, int lane)
{
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int row = r0 + i * 8 + g, col = c0 + j * 8 + 2 * q;
            if (row < nr && col < nc) out[(long long)row * ld + col] = make_double2(re[i][j][0], im[i][j][0]);
            if (row < nr && col + 1 < nc) out[(long long)row * ld + col + 1] = make_double2(re[i][j][1], im[i][j][1]);
        }
}

// Partial C tile (ta, tb) = sum over rows r of a split of conj(X[r][a]) Y[r][b].
__global__ void __launch_bounds__(128) h_gram(int n, int m, const double2* __restrict__ X,
                                              const double2* __restrict__ Y, double2* __restrict__ part, int ks, int nt)
{
    __shared__ __align__(16) HTiles t;
    const int ta = blockIdx.x / nt, tb = blockIdx.x % nt;
    const int a0 = ta * HM, b0 = tb * HM;
    const long long chunk = ((long long)n + ks - 1) / ks;
    const int r0 = (int)min((long long)n, blockIdx.y * chunk), r1 = (int)min((long long)n, (blockIdx.y + 1) * chunk);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    double re[4][4][2], im[4][4][2];
    hzero(re);
    hzero(im);
    for (int k0 = r0; k0 < r1; k0 += HK) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = tid + u * 128;
            const int kk = idx >> 6, c = idx & 63;
            const int r = k0 + kk;
            const bool rok = r < r1;
            const double2 x = (rok && a0 + c < m) ? X[(long long)r * m + a0 + c] : make_double2(0.0, 0.0);
            const double2 y = (rok && b0 + c < m) ? Y[(long long)r * m + b0 + c] : make_double2(0.0, 0.0);
            t.ar[kk][c] = x.x;
            t.ai[kk][c] = -x.y;  // conj(X)
            t.br[kk][c] = y.x;
            t.bi[kk][c] = y.y;
        }
        __syncthreads();
        htile_mma(t, re, im, wr, wc, lane);
        __syncthreads();
    }
    hstore(re, im, part + (long long)blockIdx.y * m * m, m, m, m, a0 + wr, b0 + wc, lane);
}

__global__ void h_gram_reduce(int m, const double2* __restrict__ part, int ks, double2* __restrict__ C)
{
    const long long total = (long long)m * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        for (int s = 0; s < ks; ++s) {
            const double2 u = part[(long long)s * total + idx];
            v.x += u.x;
            v.y += u.y;
        }
        C[idx] = v;
    }
}

size_t h_gram_partial(int n, int m, int* ks_out)
{
    const int nt = (m + HM - 1) / HM;
    int ks = (4 * num_sms() + nt * nt - 1) / (nt * nt);
    const int maxk = (n + 255) / 256;
    if (ks > maxk) ks = maxk;
    if (ks < 1) ks = 1;
    if (ks_out) *ks_out = ks;
    return (size_t)ks * m * m;
}

cudaError_t launch_h_gram(int n, int m, const double2* X, const double2* Y, double2* C, double2* part, int ks,
                          cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    const int nt = (m + HM - 1) / HM;
    h_gram<<<dim3(nt * nt, ks), 128, 0, s>>>(n, m, X, Y, part, ks, nt);
    long long blocks = ((long long)m * m + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    h_gram_reduce<<<(int)blocks, 256, 0, s>>>(m, part, ks, C);
    count_launches(2);
    return cudaGetLastError();
}

// C (n x k) = A (n x m) V (m x k), complex row-major.
__global__ void __launch_bounds__(128) h_gemm(int n, int m, int k, const double2* __restrict__ A,
                                              const double2* __restrict__ V, double2* __restrict__ C)
{
    __shared__ __align__(16) HTiles t;
    const int r0 = blockIdx.x * HM, c0 = blockIdx.y * HM;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    double re[4][4][2], im[4][4][2];
    hzero(re);
    hzero(im);
    for (int k0 = 0; k0 < m; k0 += HK) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = tid + u * 128;
            // A tile: 64 rows x 16 k, transposed into [k][row]
            const int ar = idx >> 4, ak = idx & 15;
            const int gr = r0 + ar, gk = k0 + ak;
            const double2 x = (gr < n && gk < m) ? A[(long long)gr * m + gk] : make_double2(0.0, 0.0);
            t.ar[ak][ar] = x.x;
            t.ai[ak][ar] = x.y;
            // V tile: 16 k x 64 cols
            const int bk = idx >> 6, bc = idx & 63;
            const int vk = k0 + bk, vc = c0 + bc;
            const double2 y = (vk < m && vc < k) ? V[(long long)vk * k + vc] : make_double2(0.0, 0.0);
            t.br[bk][bc] = y.x;
            t.bi[bk][bc] = y.y;
        }
        __syncthreads();
        htile_mma(t, re, im, wr, wc, lane);
        __syncthreads();
    }
    hstore(re, im, C, k, n, k, r0 + wr, c0 + wc, lane);
}

cudaError_t launch_h_gemm(int n, int m, int k, const double2* A, const double2* V, double2* C, cudaStream_t s)
{
    if (n <= 0 || k <= 0) return cudaSuccess;
    h_gemm<<<dim3((n + HM - 1) / HM, (k + HM - 1) / HM), 128, 0, s>>>(n, m, k, A, V, C);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- residuals
// Pass 1: per item (256 rows, 32 columns) R rows and per-column partials of
// |R|^2 and |B x|^2 -> part[rb][m][2]; pass 2: fixed-order column sums.
static constexpr int kResRB = 256;

__device__ __forceinline__ double2 row_dot_c(const int* __restrict__ ia, const int* __restrict__ ja,
                                             const double2* __restrict__ av, int i, const double2* __restrict__ X,
                                             int m, int c)
{
    double2 acc = make_double2(0.0, 0.0);
    const int s = __ldg(ia + i), e = __ldg(ia + i + 1);
    for (int k = s; k < e; ++k) {
        const double2 a = av[k], x = X[(long long)__ldg(ja + k) * m + c];
        acc.x = fma(a.x, x.x, fma(-a.y, x.y, acc.x));
        acc.y = fma(a.x, x.y, fma(a.y, x.x, acc.y));
    }
    return acc;
}

__global__ void __launch_bounds__(256) h_res_rows(int n, int m, const int* __restrict__ ia, const int* __restrict__ ja,
                                                  const double2* __restrict__ av, const int* __restrict__ ib,
                                                  const int* __restrict__ jb, const double2* __restrict__ bv,
                                                  const double2* __restrict__ X, const double* __restrict__ lam,
                                                  double2* __restrict__ R, double* __restrict__ part)
{
    __shared__ double2 sh[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nrb = (n + kResRB - 1) / kResRB, nch = (m + 31) / 32;
    for (long long it = blockIdx.x; it < (long long)nrb * nch; it += gridDim.x) {
        const int rb = (int)(it / nch), c = (int)(it % nch) * 32 + lane;
        double rr = 0.0, bb = 0.0;
        if (c < m) {
            const double l = lam[c];
            for (int i = rb * kResRB + warp; i < min(n, (rb + 1) * kResRB); i += 8) {
                const double2 ax = row_dot_c(ia, ja, av, i, X, m, c);
                const double2 bx = ib ? row_dot_c(ib, jb, bv, i, X, m, c) : X[(long long)i * m + c];
                const double2 r = make_double2(fma(-l, bx.x, ax.x), fma(-l, bx.y, ax.y));
                R[(long long)i * m + c] = r;
                rr = fma(r.x, r.x, fma(r.y, r.y, rr));
                bb = fma(bx.x, bx.x, fma(bx.y, bx.y, bb));
            }
        }
        sh[warp][lane] = make_double2(rr, bb);
        __syncthreads();
        if (warp == 0 && c < m) {
            double s1 = 0.0, s2 = 0.0;
            for (int w = 0; w < 8; ++w) {
                s1 += sh[w][lane].x;
                s2 += sh[w][lane].y;
            }
            part[((long long)rb * m + c) * 2] = s1;
            part[((long long)rb * m + c) * 2 + 1] = s2;
        }
        __syncthreads();
    }
}

__global__ void h_res_cols(int n, int m, const double* __restrict__ part, double alpha, double* __restrict__ res)
{
    __shared__ double s1[256], s2[256];
    const int nrb = (n + kResRB - 1) / kResRB, c = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int rb = threadIdx.x; rb < nrb; rb += blockDim.x) {
        a += part[((long long)rb * m + c) * 2];
        b += part[((long long)rb * m + c) * 2 + 1];
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double rn = sqrt(s1[0]), bn = sqrt(s2[0]);
        res[c] = bn > 0.0 ? rn / (alpha * bn) : 0.0;
    }
}

size_t h_resid_partial(int n, int m) { return (size_t)((n + kResRB - 1) / kResRB) * m * 2; }

cudaError_t launch_h_residual(int n, int m, const int* ia, const int* ja, const double2* av, const int* ib,
                              const int* jb, const double2* bv, const double2* X, const double* lam, double2* R,
                              double* part, double* res, double alpha, cudaStream_t s)
{
    if (n <= 0 || m <= 0) return cudaSuccess;
    const long long items = (long long)((n + kResRB - 1) / kResRB) * ((m + 31) / 32);
    const long long cap = (long long)num_sms() * 8;
    h_res_rows<<<(int)(items < cap ? items : cap), 256, 0, s>>>(n, m, ia, ja, av, ib, jb, bv, X, lam, R, part);
    h_res_cols<<<m, 256, 0, s>>>(n, m, part, alpha, res);
    count_launches(2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- sliced products through real views
// A row-major n x m complex block is, viewed as doubles, the real n x 2m block
// Z = [Re q_1, Im q_1, Re q_2, ...].  Its real Gram G = Z^T Z' (2m x 2m, by the
// sliced BF16 kernel) holds every product of real and imaginary parts, and
//   (Q^H Y)[a][b] = (G[2a][2b] + G[2a+1][2b+1]) + i (G[2a][2b+1] - G[2a+1][2b]).
// Likewise X = Q V is the real product Z W with W[2a][2b] = W[2a+1][2b+1] =
// Re v_ab, W[2a][2b+1] = Im v_ab, W[2a+1][2b] = -Im v_ab, which leaves X in
// the same interleaved layout.
__global__ void h_from_real_gram(int m, const double* __restrict__ G, double2* __restrict__ C)
{
    const long long total = (long long)m * m;
    const size_t ld = 2 * (size_t)m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(idx / m), b = (int)(idx % m);
        const double rr = G[(2 * a) * ld + 2 * b], ii = G[(2 * a + 1) * ld + 2 * b + 1];
        const double ri = G[(2 * a) * ld + 2 * b + 1], ir = G[(2 * a + 1) * ld + 2 * b];
        C[idx] = make_double2(rr + ii, ri - ir);
    }
}

__global__ void h_real_coupling(int m, int k, const double2* __restrict__ V, double* __restrict__ W)
{
    const long long total = (long long)m * k;
    const size_t ld = 2 * (size_t)k;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(idx / k), b = (int)(idx % k);
        const double2 v = V[idx];
        W[(2 * a) * ld + 2 * b] = v.x;
        W[(2 * a) * ld + 2 * b + 1] = v.y;
        W[(2 * a + 1) * ld + 2 * b] = -v.y;
        W[(2 * a + 1) * ld + 2 * b + 1] = v.x;
    }
}

// split-K partials of either Gram form (the upper-triangle form takes more splits)
static size_t h_sliced_part_doubles(int n, int m2)
{
    return std::max(gram_oz_partial_doubles(n, m2, nullptr, nullptr, num_sms(), true),
                    gram_oz_partial_doubles(n, m2, nullptr, nullptr, num_sms(), false));
}

static size_t r256(size_t b) { return (b + 255) / 256 * 256; }

// the pieces of h_sliced_carve, each rounded up to 256 bytes
size_t h_sliced_work_bytes(int n, int m)
{
    const int m2 = 2 * m;
    return r256(h_sliced_part_doubles(n, m2) * sizeof(double)) + 2 * r256((size_t)m2 * m2 * sizeof(double)) +
           r256(gram_oz_work_bytes(m2)) + r256(gemm_oz_work_bytes(n, m2, m2)) + 256;
}

static void h_sliced_carve(int n, int m, void* work, double** part, double** G, double** W, int** ex, void** gw)
{
    const int m2 = 2 * m;
    char* p = (char*)work;
    auto take = [&](size_t bytes) { char* q = p; p += r256(bytes); return q; };
    *part = (double*)take(h_sliced_part_doubles(n, m2) * sizeof(double));
    *G = (double*)take((size_t)m2 * m2 * sizeof(double));
    *W = (double*)take((size_t)m2 * m2 * sizeof(double));
    *ex = (int*)take(gram_oz_work_bytes(m2));
    *gw = take(gemm_oz_work_bytes(n, m2, m2));
}

cudaError_t launch_h_gram_sliced(int n, int m, const double2* X, const double2* Y, double2* C, void* work,
                                 cudaStream_t s)
{
    double *part, *G, *W;
    int* ex;
    void* gw;
    h_sliced_carve(n, m, work, &part, &G, &W, &ex, &gw);
    // X = Y: the real Gram is symmetric and its upper triangle suffices
    cudaError_t e = launch_gram_oz(n, 2 * m, (const double*)X, (const double*)Y, G, part, ex, s, X != Y);
    if (e != cudaSuccess) return e;
    const long long mm = (long long)m * m;
    h_from_real_gram<<<(int)std::min<long long>((mm + 255) / 256, 1024), 256, 0, s>>>(m, G, C);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_h_gemm_sliced(int n, int m, int k, const double2* A, const double2* V, double2* C, void* work,
                                 cudaStream_t s)
{
    double *part, *G, *W;
    int* ex;
    void* gw;
    h_sliced_carve(n, std::max(m, k), work, &part, &G, &W, &ex, &gw);
    const long long mk = (long long)m * k;
    h_real_coupling<<<(int)std::min<long long>((mk + 255) / 256, 1024), 256, 0, s>>>(m, k, V, W);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_gemm_oz(n, 2 * m, 2 * k, (const double*)A, W, (double*)C, gw, s);
}

// ---------------------------------------------------------------- Hermitian Jacobi (one CTA)
// Cyclic Jacobi with the round-robin (circle) ordering: in each of the N - 1
// rounds of a sweep (N = size rounded up to even) the N / 2 index pairs are
// disjoint, so all their rotations are computed from the same matrix and
// applied together (columns, then rows).  The rotation of a pair (p, q) with
// a_pq = |a_pq| e: D = diag(1, conj e) makes the pair's 2 x 2 block real,
// then the real rotation with t = tan(theta) the smaller root of
// t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 |a_pq|), annihilates it;
// J = D R has columns (c, -s conj e) and (s, c conj e) on rows (p, q).
// A pair is skipped when |a_pq| <= max(1.1e-16 sqrt|a_pp a_qq|, 1e-18 ||A||_F);
// the sweeps stop when a sweep rotates nothing, or after kHJSweeps.
static constexpr int kHJMax = 1024;
static constexpr int kHJSweeps = 60;

// size = *kdev when kdev is set (else m); A and Vout have leading dimension ld.
// Vout gets the eigenvectors in ascending order of lam (zero outside size x size).
__global__ void __launch_bounds__(1024) h_jacobi(int m, int ld, const int* __restrict__ kdev, double2* __restrict__ A,
                                                 double2* __restrict__ Vw, double* __restrict__ lam,
                                                 double2* __restrict__ Vout, int* __restrict__ status)
{
    __shared__ double s_c[kHJMax / 2], s_s[kHJMax / 2];
    __shared__ double2 s_e[kHJMax / 2];
    __shared__ int s_p[kHJMax / 2], s_q[kHJMax / 2], s_on[kHJMax / 2];
    __shared__ double s_red[32];
    __shared__ int s_rot;
    const int tid = threadIdx.x, nt = blockDim.x;
    int n = kdev ? *kdev : m;
    if (n > m) n = m;
    if (n < 0) n = 0;
    const int N = (n + 1) & ~1, half = N / 2;
    for (long long idx = tid; idx < (long long)n * n; idx += nt) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        Vw[(long long)i * ld + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    // Frobenius norm (fixed-order block reduction)
    double f = 0.0;
    for (long long idx = tid; idx < (long long)n * n; idx += nt) {
        const double2 v = A[(idx / n) * ld + idx % n];
        f = fma(v.x, v.x, fma(v.y, v.y, f));
    }
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = f;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (nt + 31) / 32; ++w) t += s_red[w];
        s_red[0] = t;
    }
    __syncthreads();
    const double absfloor = 1e-18 * sqrt(s_red[0]);
    int sweep = 0;
    bool more = n > 1;
    while (more && sweep < kHJSweeps) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < N - 1; ++r) {
            // pairs of round r: (r, N-1) and ((r+k) mod (N-1), (r-k) mod (N-1))
            for (int k = tid; k < half; k += nt) {
                int p, q;
                if (k == 0) {
                    p = r;
                    q = N - 1;
                } else {
                    p = (r + k) % (N - 1);
                    q = (r - k + (N - 1)) % (N - 1);
                }
                if (p > q) { const int t = p; p = q; q = t; }
                int on = 0;
                double c = 1.0, s = 0.0;
                double2 e = make_double2(1.0, 0.0);
                if (q < n) {
                    const double2 apq = A[(long long)p * ld + q];
                    const double mag = hypot(apq.x, apq.y);
                    const double app = A[(long long)p * ld + p].x, aqq = A[(long long)q * ld + q].x;
                    const double thr = fmax(1.1e-16 * sqrt(fabs(app * aqq)), absfloor);
                    if (mag > thr) {
                        on = 1;
                        e = make_double2(apq.x / mag, apq.y / mag);
                        const double tau = (aqq - app) / (2.0 * mag);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                s_p[k] = p;
                s_q[k] = q;
                s_on[k] = on;
                s_c[k] = c;
                s_s[k] = s;
                s_e[k] = e;
                if (on) atomicAdd(&s_rot, 1);
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (long long idx = tid; idx < (long long)half * n; idx += nt) {
                const int k = (int)(idx / n), i = (int)(idx % n);
                if (!s_on[k]) continue;
                const int p = s_p[k], q = s_q[k];
                const double c = s_c[k], s = s_s[k];
                const double2 ec = make_double2(s_e[k].x, -s_e[k].y);
                double2* rows[2] = {A, Vw};
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    double2* M = rows[w];
                    const double2 xp = M[(long long)i * ld + p], xq = M[(long long)i * ld + q];
                    const double2 exq = make_double2(ec.x * xq.x - ec.y * xq.y, ec.x * xq.y + ec.y * xq.x);
                    M[(long long)i * ld + p] = make_double2(c * xp.x - s * exq.x, c * xp.y - s * exq.y);
                    M[(long long)i * ld + q] = make_double2(s * xp.x + c * exq.x, s * xp.y + c * exq.y);
                }
            }
            __syncthreads();
            // rows: A <- J^H A
            for (long long idx = tid; idx < (long long)half * n; idx += nt) {
                const int k = (int)(idx / n), j = (int)(idx % n);
                if (!s_on[k]) continue;
                const int p = s_p[k], q = s_q[k];
                const double c = s_c[k], s = s_s[k];
                const double2 e = s_e[k];
                const double2 yp = A[(long long)p * ld + j], yq = A[(long long)q * ld + j];
                const double2 eyq = make_double2(e.x * yq.x - e.y * yq.y, e.x * yq.y + e.y * yq.x);
                A[(long long)p * ld + j] = make_double2(c * yp.x - s * eyq.x, c * yp.y - s * eyq.y);
                A[(long long)q * ld + j] = make_double2(s * yp.x + c * eyq.x, s * yp.y + c * eyq.y);
            }
            __syncthreads();
            for (int k = tid; k < half; k += nt)
                if (s_on[k]) {
                    const int p = s_p[k], q = s_q[k];
                    A[(long long)p * ld + q] = make_double2(0.0, 0.0);
                    A[(long long)q * ld + p] = make_double2(0.0, 0.0);
                    A[(long long)p * ld + p].y = 0.0;
                    A[(long long)q * ld + q].y = 0.0;
                }
            __syncthreads();
        }
        more = s_rot > 0;
        ++sweep;
        __syncthreads();
    }
    // ascending order: rank by value, ties by index
    __shared__ int s_rank[kHJMax];
    for (int i = tid; i < n; i += nt) {
        const double li = A[(long long)i * ld + i].x;
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const double lj = A[(long long)j * ld + j].x;
            rk += (lj < li) || (lj == li && j < i);
        }
        s_rank[i] = rk;
        lam[rk] = li;
    }
    for (int i = n + tid; i < m; i += nt) lam[i] = 0.0;
    __syncthreads();
    for (long long idx = tid; idx < (long long)m * m; idx += nt) {
        const int r = (int)(idx / m), c = (int)(idx % m);
        Vout[(long long)r * ld + c] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (long long idx = tid; idx < (long long)n * n; idx += nt) {
        const int r = (int)(idx / n), i = (int)(idx % n);
        Vout[(long long)r * ld + s_rank[i]] = Vw[(long long)r * ld + i];
    }
    if (tid == 0) *status = more ? -1 : 0;
}

cudaError_t launch_h_jacobi(int m, double2* A, double2* Vw, double* lam, double2* V, const int* kdev, int* status_dev,
                            cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    if (m > kHJMax) return cudaErrorInvalidValue;
    h_jacobi<<<1, 1024, 0, s>>>(m, m, kdev, A, Vw, lam, V, status_dev);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Hermitian Jacobi (many CTAs)
// The same rotations as h_jacobi, spread over the CTAs of one cooperative
// launch with one grid barrier per round (GB300's FP64 rate per SM is low, so
// one CTA is slow): every CTA computes all rotations of the round (identical
// inputs and code, so identical angles) into shared memory, then updates its
// share of the 2 x 2 blocks from the current copy of A into the other copy,
// so no CTA writes what another still reads.  Block (k, l) holds rows p_k, q_k
// and columns p_l, q_l; with J_k = D_k R_k (columns (c, -s conj e) and
// (s, c conj e)) it becomes J_k^H A J_l; a diagonal block becomes
// diag(a_pp - t |a_pq|, a_qq + t |a_pq|).  The barrier spins at most
// wait_limit_cycles() cycles, then every CTA returns and *err is set.
struct HJWork {
    unsigned long long count;  // barrier arrivals since launch; never reset
    int err;
    int sweeps;
    int status;
    int pad;
    double fro;
};

__device__ __forceinline__ bool h_grid_sync(HJWork* w, long long limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = (*(volatile int*)&w->err == 0);
        if (good) {
            unsigned long long old;
            asm volatile("atom.add.release.gpu.u64 %0, [%1], 1;" : "=l"(old) : "l"(&w->count) : "memory");
            const unsigned long long target = (old / gridDim.x + 1) * gridDim.x;
            const long long t0 = clock64();
            for (;;) {
                unsigned long long cur;
                asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(cur) : "l"(&w->count) : "memory");
                if (cur >= target) break;
                if (*(volatile int*)&w->err) { good = 0; break; }
                if (clock64() - t0 > limit) {
                    atomicExch(&w->err, 1);
                    good = 0;
                    break;
                }
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__global__ void __launch_bounds__(256) h_jacobi_coop(int m, double2* __restrict__ A, double2* __restrict__ A2,
                                                     double2* __restrict__ Vw, double* __restrict__ lam,
                                                     double2* __restrict__ Vout, HJWork* __restrict__ w,
                                                     long long limit)
{
    __shared__ double s_c[kHJMax / 2], s_s[kHJMax / 2], s_t[kHJMax / 2];
    __shared__ double2 s_e[kHJMax / 2];
    __shared__ int s_p[kHJMax / 2], s_q[kHJMax / 2];
    __shared__ double s_red[8];
    __shared__ int s_any;
    const int N = (m + 1) & ~1, half = N / 2;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
    for (long long idx = gtid; idx < (long long)m * m; idx += gsz)
        Vw[idx] = make_double2(idx / m == idx % m ? 1.0 : 0.0, 0.0);
    if (blockIdx.x == 0) {  // Frobenius norm, fixed order
        double f = 0.0;
        for (long long idx = threadIdx.x; idx < (long long)m * m; idx += blockDim.x) {
            const double2 v = A[idx];
            f = fma(v.x, v.x, fma(v.y, v.y, f));
        }
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = f;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_red[i];
            w->fro = sqrt(t);
        }
    }
    if (!h_grid_sync(w, limit)) return;
    const double absfloor = 1e-18 * *(volatile double*)&w->fro;
    double2* cur = A;
    double2* nxt = A2;
    int sweep = 0;
    bool more = m > 1;
    while (more && sweep < kHJSweeps) {
        if (threadIdx.x == 0) s_any = 0;
        __syncthreads();
        for (int r = 0; r < N - 1; ++r) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int p, q;
                if (k == 0) {
                    p = r;
                    q = N - 1;
                } else {
                    p = (r + k) % (N - 1);
                    q = (r - k + (N - 1)) % (N - 1);
                }
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0, tt = 0.0;
                double2 e = make_double2(1.0, 0.0);
                if (q < m) {
                    const double2 apq = __ldcg(cur + (size_t)p * m + q);
                    const double mag = hypot(apq.x, apq.y);
                    const double app = __ldcg(cur + (size_t)p * m + p).x, aqq = __ldcg(cur + (size_t)q * m + q).x;
                    const double thr = fmax(1.1e-16 * sqrt(fabs(app * aqq)), absfloor);
                    if (mag > thr) {
                        e = make_double2(apq.x / mag, apq.y / mag);
                        const double tau = (aqq - app) / (2.0 * mag);
                        tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                        s_any = 1;
                    }
                }
                s_c[k] = c;
                s_s[k] = s;
                s_t[k] = tt;
                s_e[k] = e;
                s_p[k] = p;
                s_q[k] = q;
            }
            __syncthreads();
            for (long long idx = gtid; idx < (long long)half * half; idx += gsz) {
                const int k = (int)(idx / half), l = (int)(idx % half);
                const int p = s_p[k], q = s_q[k], pp = s_p[l], qq = s_q[l];
                const bool qv = q < m, qqv = qq < m;
                if (k == l) {
                    const double2 app = __ldcg(cur + (size_t)p * m + p);
                    if (!qv) {
                        nxt[(size_t)p * m + p] = make_double2(app.x, 0.0);
                        continue;
                    }
                    const double2 apq = __ldcg(cur + (size_t)p * m + q), aqq = __ldcg(cur + (size_t)q * m + q);
                    if (s_s[k] == 0.0) {
                        nxt[(size_t)p * m + p] = make_double2(app.x, 0.0);
                        nxt[(size_t)q * m + q] = make_double2(aqq.x, 0.0);
                        nxt[(size_t)p * m + q] = apq;
                        nxt[(size_t)q * m + p] = __ldcg(cur + (size_t)q * m + p);
                    } else {
                        const double mag = hypot(apq.x, apq.y);
                        nxt[(size_t)p * m + p] = make_double2(app.x - s_t[k] * mag, 0.0);
                        nxt[(size_t)q * m + q] = make_double2(aqq.x + s_t[k] * mag, 0.0);
                        nxt[(size_t)p * m + q] = make_double2(0.0, 0.0);
                        nxt[(size_t)q * m + p] = make_double2(0.0, 0.0);
                    }
                    continue;
                }
                const double ck = s_c[k], sk = s_s[k], cl = s_c[l], sl = s_s[l];
                const double2 ek = s_e[k], el = s_e[l];
                const double2 z = make_double2(0.0, 0.0);
                const double2 x00 = __ldcg(cur + (size_t)p * m + pp);
                const double2 x01 = qqv ? __ldcg(cur + (size_t)p * m + qq) : z;
                const double2 x10 = qv ? __ldcg(cur + (size_t)q * m + pp) : z;
                const double2 x11 = (qv && qqv) ? __ldcg(cur + (size_t)q * m + qq) : z;
                // rows (J_k^H): y0 = c x0 - s e x1, y1 = s x0 + c e x1
                const double2 ex10 = make_double2(ek.x * x10.x - ek.y * x10.y, ek.x * x10.y + ek.y * x10.x);
                const double2 ex11 = make_double2(ek.x * x11.x - ek.y * x11.y, ek.x * x11.y + ek.y * x11.x);
                const double2 y00 = make_double2(ck * x00.x - sk * ex10.x, ck * x00.y - sk * ex10.y);
                const double2 y01 = make_double2(ck * x01.x - sk * ex11.x, ck * x01.y - sk * ex11.y);
                const double2 y10 = make_double2(sk * x00.x + ck * ex10.x, sk * x00.y + ck * ex10.y);
                const double2 y11 = make_double2(sk * x01.x + ck * ex11.x, sk * x01.y + ck * ex11.y);
                // columns (J_l): col p' = c y.0 - s conj(e) y.1, col q' = s y.0 + c conj(e) y.1
                const double2 ec = make_double2(el.x, -el.y);
                const double2 ey01 = make_double2(ec.x * y01.x - ec.y * y01.y, ec.x * y01.y + ec.y * y01.x);
                const double2 ey11 = make_double2(ec.x * y11.x - ec.y * y11.y, ec.x * y11.y + ec.y * y11.x);
                nxt[(size_t)p * m + pp] = make_double2(cl * y00.x - sl * ey01.x, cl * y00.y - sl * ey01.y);
                if (qqv) nxt[(size_t)p * m + qq] = make_double2(sl * y00.x + cl * ey01.x, sl * y00.y + cl * ey01.y);
                if (qv) nxt[(size_t)q * m + pp] = make_double2(cl * y10.x - sl * ey11.x, cl * y10.y - sl * ey11.y);
                if (qv && qqv)
                    nxt[(size_t)q * m + qq] = make_double2(sl * y10.x + cl * ey11.x, sl * y10.y + cl * ey11.y);
            }
            for (long long idx = gtid; idx < (long long)m * half; idx += gsz) {  // V <- V J
                const int i = (int)(idx / half), k = (int)(idx % half);
                const double sk = s_s[k];
                if (sk == 0.0) continue;
                const double ck = s_c[k];
                const double2 ec = make_double2(s_e[k].x, -s_e[k].y);
                const int p = s_p[k], q = s_q[k];
                const double2 vp = Vw[(size_t)i * m + p], vq = Vw[(size_t)i * m + q];
                const double2 evq = make_double2(ec.x * vq.x - ec.y * vq.y, ec.x * vq.y + ec.y * vq.x);
                Vw[(size_t)i * m + p] = make_double2(ck * vp.x - sk * evq.x, ck * vp.y - sk * evq.y);
                Vw[(size_t)i * m + q] = make_double2(sk * vp.x + ck * evq.x, sk * vp.y + ck * evq.y);
            }
            if (!h_grid_sync(w, limit)) return;
            double2* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        more = s_any != 0;  // same decision in every CTA
        ++sweep;
    }
    for (int i = gtid; i < m; i += gsz) {  // ascending order: rank by value, ties by index
        const double li = __ldcg(cur + (size_t)i * m + i).x;
        int rk = 0;
        for (int j = 0; j < m; ++j) {
            const double lj = __ldcg(cur + (size_t)j * m + j).x;
            rk += (lj < li) || (lj == li && j < i);
        }
        lam[rk] = li;
        for (int row = 0; row < m; ++row) Vout[(size_t)row * m + rk] = Vw[(size_t)row * m + i];
    }
    if (gtid == 0) {
        w->sweeps = sweep;
        w->status = more ? -1 : 0;
    }
}

size_t h_jacobi_coop_bytes(int m) { return 2 * (size_t)m * m * sizeof(double2) + sizeof(HJWork) + 512; }

// A (m x m) is overwritten; V gets the eigenvectors in ascending order of
// lam.  *status_dev: 0, -1 (sweep limit) or -2 (grid barrier timed out).
// Returns a CUDA error, cudaSuccess otherwise.
__global__ void h_coop_status(const HJWork* w, int* status) { *status = w->err ? -2 : w->status; }

static cudaError_t launch_h_jacobi_coop(int m, double2* A, double* lam, double2* V, void* work, int* status_dev,
                                        cudaStream_t s)
{
    char* p = (char*)work;
    HJWork* w = (HJWork*)p;
    double2* A2 = (double2*)(p + 256);
    double2* Vw = A2 + (size_t)m * m;
    cudaError_t e = cudaMemsetAsync(w, 0, sizeof(HJWork), s);
    if (e != cudaSuccess) return e;
    static const int per_sm = [] {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, h_jacobi_coop, 256, 0);
        return v > 0 ? v : 1;
    }();
    const int half = (m + 1) / 2;
    long long blocks = ((long long)m * half + 255) / 256;
    const long long cap = std::min<long long>((long long)num_sms() * per_sm, num_sms());
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    long long limit = wait_limit_cycles();
    void* args[] = {&m, &A, &A2, &Vw, &lam, &V, &w, &limit};
    e = cudaLaunchCooperativeKernel((void*)h_jacobi_coop, dim3((unsigned)blocks), dim3(256), args, 0, s);
    count_launches(1);
    if (e != cudaSuccess) return e;
    // status: -2 when the barrier gave up, -1 at the sweep limit, else 0
    h_coop_status<<<1, 1, 0, s>>>(w, status_dev);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reduced generalized problem
// Aq v = lambda Bq v, both symmetrised as (M + M^H)/2.  Scaling D =
// diag(Bq)^{-1/2}; Jacobi on D Bq D = U diag(d) U^H; keep d > 1e-14 max d
// (k of them); S = D U_k d_k^{-1/2} (B-orthonormal basis of the kept space);
// Jacobi on S^H Aq S = W Lambda W^H; V = S W.
__global__ void h_rg_prep(int m, const double2* __restrict__ Aq, const double2* __restrict__ Bq, double2* __restrict__ As,
                          double2* __restrict__ Bs)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)m * m;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / m), j = (int)(idx % m);
        const double bi = Bq[(long long)i * m + i].x, bj = Bq[(long long)j * m + j].x;
        const double di = bi > 0.0 ? 1.0 / sqrt(bi) : 0.0, dj = bj > 0.0 ? 1.0 / sqrt(bj) : 0.0;
        const double2 b1 = Bq[idx], b2 = Bq[(long long)j * m + i];
        const double2 a1 = Aq[idx], a2 = Aq[(long long)j * m + i];
        Bs[idx] = make_double2(0.5 * (b1.x + b2.x) * di * dj, 0.5 * (b1.y - b2.y) * di * dj);
        As[idx] = make_double2(0.5 * (a1.x + a2.x), 0.5 * (a1.y - a2.y));
    }
}

// One CTA: k = #{d > 1e-14 max d}; S[:, c] = D U[:, m-1-c] / sqrt(d[m-1-c]), c < k.
__global__ void __launch_bounds__(1024) h_rg_form_s(int m, const double2* __restrict__ Bq, const double* __restrict__ d,
                                                    const double2* __restrict__ U, double2* __restrict__ S,
                                                    int* __restrict__ mk, int* __restrict__ status)
{
    __shared__ int s_k;
    if (threadIdx.x == 0) {
        const double dmax = d[m - 1];  // ascending
        int k = 0;
        if (dmax > 0.0)
            for (int i = m - 1; i >= 0 && d[i] > 1e-14 * dmax; --i) ++k;
        s_k = k;
        *mk = k;
        if (k == 0) *status = -3;
    }
    __syncthreads();
    const int k = s_k;
    for (long long idx = threadIdx.x; idx < (long long)m * m; idx += blockDim.x) {
        const int r = (int)(idx / m), c = (int)(idx % m);
        double2 v = make_double2(0.0, 0.0);
        if (c < k) {
            const int i = m - 1 - c;
            const double br = Bq[(long long)r * m + r].x;
            const double f = (br > 0.0 ? 1.0 / sqrt(br) : 0.0) / sqrt(d[i]);
            const double2 u = U[(long long)r * m + i];
            v = make_double2(f * u.x, f * u.y);
        }
        S[idx] = v;
    }
}

// C <- (C + C^H) / 2 in place (thread per pair i <= j).
__global__ void h_herm_part(int m, double2* __restrict__ C)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)m * m;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / m), j = (int)(idx % m);
        if (i > j) continue;
        const double2 a = C[idx], b = C[(long long)j * m + i];
        const double2 s = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        C[idx] = s;
        C[(long long)j * m + i] = make_double2(s.x, -s.y);
    }
}

// Cholesky route (the LAPACK hegv family's first step, as on the real path):
// one CTA factors the scaled Bs = D Bq D = L L^H in the global scratch G
// (row-major, lower triangle read), inverts X = L^{-1}, and writes the
// B-orthonormal basis S = D X^H (upper triangular: S[r][c] = d_r conj(X[c][r])).
// status = 0 when every pivot is positive and ||X||_F^2 <= 1e8, else 1 (then
// the two-Jacobi route is taken).  After the first loops Bs is close to I, so
// S^H Aq S is close to diagonal and its Jacobi converges in a few sweeps.
static constexpr double kHCholCondMax = 1e8;

__global__ void __launch_bounds__(1024) h_rg_cholinv(int m, const double2* __restrict__ Bs, const double2* __restrict__ Bq,
                                                     double2* __restrict__ G, double* __restrict__ xd,
                                                     double2* __restrict__ cj, double2* __restrict__ S,
                                                     int* __restrict__ status, int* __restrict__ mk)
{
    __shared__ double red[32];
    __shared__ int s_ok;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (long long idx = tid; idx < (long long)m * m; idx += nt) G[idx] = Bs[idx];
    if (tid == 0) s_ok = 1;
    __syncthreads();
    for (int j = 0; j < m; ++j) {  // right-looking: two barriers per column
        const double dj = G[(size_t)j * m + j].x;
        if (!(dj > 0.0)) {  // same value in every thread: uniform exit
            if (tid == 0) *status = 1;
            return;
        }
        const double l = sqrt(dj);
        for (int i = j + 1 + tid; i < m; i += nt) {
            const double2 g = G[(size_t)i * m + j];
            const double2 v = make_double2(g.x / l, g.y / l);
            G[(size_t)i * m + j] = v;
            cj[i] = v;
        }
        if (tid == 0) xd[j] = l;
        __syncthreads();
        for (int i = j + 1 + warp; i < m; i += nw) {  // G[i][k] -= cj[i] conj(cj[k]), j < k <= i
            const double2 ci = cj[i];
            for (int k = j + 1 + lane; k <= i; k += 32) {
                const double2 ck = cj[k];
                double2& g = G[(size_t)i * m + k];
                g.x -= ci.x * ck.x + ci.y * ck.y;
                g.y -= ci.y * ck.x - ci.x * ck.y;
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < m; i += nt) {
        const double l = xd[i];
        G[(size_t)i * m + i] = make_double2(l, 0.0);
        xd[i] = 1.0 / l;
    }
    __syncthreads();
    // X = L^{-1}: warp w owns columns c = w, w + nw, ...; X[i][c] =
    // -(1/L_ii) sum_{c <= k < i} L[i][k] X[k][c], stored at G[c][i] (c < i)
    double nrm = 0.0;
    for (int c = warp; c < m; c += nw) {
        const double xc = xd[c];
        if (lane == 0) nrm += xc * xc;
        for (int i = c + 1; i < m; ++i) {
            double2 s = make_double2(0.0, 0.0);
            for (int k = c + lane; k < i; k += 32) {
                const double2 lik = G[(size_t)i * m + k];
                const double2 xk = k == c ? make_double2(xc, 0.0) : G[(size_t)c * m + k];
                s.x += lik.x * xk.x - lik.y * xk.y;
                s.y += lik.x * xk.y + lik.y * xk.x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            }
            const double2 v = make_double2(-s.x * xd[i], -s.y * xd[i]);
            if (lane == 0) {
                G[(size_t)c * m + i] = v;
                nrm += v.x * v.x + v.y * v.y;
            }
            __syncwarp();
        }
    }
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (lane == 0) red[warp] = nrm;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[w];
        s_ok = t <= kHCholCondMax;
        *status = s_ok ? 0 : 1;
        if (s_ok) *mk = m;
    }
    __syncthreads();
    if (!s_ok) return;
    for (long long idx = tid; idx < (long long)m * m; idx += nt) {
        const int r = (int)(idx / m), c = (int)(idx % m);
        const double br = Bq[(size_t)r * m + r].x;
        const double dr = br > 0.0 ? 1.0 / sqrt(br) : 0.0;
        double2 v = make_double2(0.0, 0.0);
        if (c > r) {
            const double2 x = G[idx];  // X[c][r]
            v = make_double2(dr * x.x, -dr * x.y);
        } else if (c == r) {
            v = make_double2(dr * xd[r], 0.0);
        }
        S[idx] = v;
    }
}

size_t h_reduced_work_bytes(int m)
{
    const size_t mm = (size_t)m * m;
    int ks = 1;
    const size_t gp = h_gram_partial(m, m, &ks);
    return (9 * mm + gp + m) * sizeof(double2) + 3 * (size_t)m * sizeof(double) + 512 + h_jacobi_coop_bytes(m) + 256;
}

int h_reduced_gev(int m, const double2* Aq, const double2* Bq, double* lam, double2* V, int* mk_dev, int* status_dev,
                  void* work, cudaStream_t s)
{
    if (m <= 0 || m > kHJMax) return -1;
    const size_t mm = (size_t)m * m;
    int ks = 1;
    h_gram_partial(m, m, &ks);
    double2* As = (double2*)work;
    double2* Bs = As + mm;
    double2* U = Bs + mm;
    double2* Vw = U + mm;
    double2* S = Vw + mm;
    double2* AS = S + mm;
    double2* C = AS + mm;
    double2* W = C + mm;
    double2* gp = W + mm;
    double* d = (double*)(gp + (size_t)ks * mm);
    double2* G = (double2*)(d + m + (m & 1));  // Cholesky scratch (m x m) and column buffer (m), 16-byte aligned
    double2* cj = G + mm;
    double* xd = (double*)(cj + m);
    void* jw = (void*)(((uintptr_t)(xd + m) + 255) & ~(uintptr_t)255);  // cooperative Jacobi work
    cudaError_t e = cudaMemsetAsync(status_dev, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return -4;
    const int blocks = (int)(((long long)mm + 255) / 256 < 1024 ? ((long long)mm + 255) / 256 : 1024);
    h_rg_prep<<<blocks, 256, 0, s>>>(m, Aq, Bq, As, Bs);
    h_rg_cholinv<<<1, 1024, 0, s>>>(m, Bs, Bq, G, xd, cj, S, status_dev, mk_dev);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return -4;
    int chol = 1;
    if (cudaMemcpyAsync(&chol, status_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -4;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -4;
    if (chol == 0) {  // S^H Aq S, one Jacobi, V = S W
        if ((e = launch_h_gemm(m, m, m, As, S, AS, s)) != cudaSuccess) return -4;
        if ((e = launch_h_gram(m, m, S, AS, C, gp, ks, s)) != cudaSuccess) return -4;
        h_herm_part<<<blocks, 256, 0, s>>>(m, C);
        count_launches(1);
        if ((e = launch_h_jacobi_coop(m, C, lam, W, jw, status_dev + 1, s)) != cudaSuccess) return -4;
        if ((e = launch_h_gemm(m, m, m, S, W, V, s)) != cudaSuccess) return -4;
        return cudaGetLastError() == cudaSuccess ? 0 : -4;
    }
    if ((e = cudaMemsetAsync(status_dev, 0, sizeof(int), s)) != cudaSuccess) return -4;
    if ((e = launch_h_jacobi_coop(m, Bs, d, U, jw, status_dev, s)) != cudaSuccess) return -4;
    h_rg_form_s<<<1, 1024, 0, s>>>(m, Bq, d, U, S, mk_dev, status_dev);
    count_launches(1);
    if ((e = launch_h_gemm(m, m, m, As, S, AS, s)) != cudaSuccess) return -4;
    if ((e = launch_h_gram(m, m, S, AS, C, gp, ks, s)) != cudaSuccess) return -4;
    h_herm_part<<<blocks, 256, 0, s>>>(m, C);
    count_launches(1);
    if ((e = launch_h_jacobi(m, C, Vw, lam, W, mk_dev, status_dev + 1, s)) != cudaSuccess) return -4;
    if ((e = launch_h_gemm(m, m, m, S, W, V, s)) != cudaSuccess) return -4;
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

}  // namespace herm
}  // namespace feast
