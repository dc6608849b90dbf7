// Contour filter kernels: batched complex-shifted CSR SpMM, column-batched
// COCG for the complex symmetric systems (z_e B - A) y = rhs, and the fused
// accumulation of the quadrature sum into the FP64 subspace block Q.
//
// Method (FEAST v4.0 guide, Sec. 1.2 and the tips of Sec. 2.2): for the Ne
// half-contour nodes z_e with weights w_e, the filter is
//   Q = sum_e Re( w_e (z_e B - A)^{-1} B Y )                       (first pass)
// and, in the residual-inverse form used by every later pass,
//   Q = X diag(rho(lambda)) + sum_e Re( w_e/(z_e - lambda_j) Y_e ),
//   (z_e B - A) Y_e = A X - B X Lambda,  rho(l) = sum_e Re(w_e/(z_e - l)).
// Both are "solve, then accumulate Re(c_{e,j} y_{e,j})" with a per-column
// coefficient c, so one COCG kernel pair serves both.  Because the solution
// y = sum_k alpha_k p_k is only ever needed inside that sum, the solution
// vectors are never stored: every step adds Re(c alpha_k p_k) to Q directly.
//
// Data layout in HBM.  Subspace columns are split into groups of mt columns;
// a group tile holds, for every row, W = mt * nbp complex values ordered
// (column, node) with the node fastest, so one warp (W = 32) or half warp
// (W = 16) reads one row of a tile as a single contiguous 256-byte segment.
// Tiles are [group][row][W]; a work item is RB rows of one group tile.
// Items of one group are contiguous and groups follow each other, so the rows
// that concurrently running CTAs gather from stay inside one tile (L2 reuse).
//
// One COCG iteration is two launches:
//   A: p_k = r_k + beta p_{k-1} (computed on the fly for every gathered row),
//      q = (zB - A) p_k, write p_k, partial sums of p_k^T q;
//      the last item of a group reduces them and sets alpha = rho / p^T q.
//   B: recompute q from p_k, r -= alpha q, Q += Re(c alpha p_k),
//      partial sums of r^T r and |r|^2; the last item sets beta and the
//      convergence state of each column.
// Recomputing q instead of storing it saves a full write+read of the block
// vector; the matrix itself is a few MB and stays in L2.
// Reductions are deterministic: fixed per-thread order, fixed block order, and
// the partials of a group are summed in item order by whichever CTA finishes
// the group last.
#include "feast_internal.cuh"

namespace feast {

static constexpr int kThreads = 256;
static constexpr int kPartStride = 4;
#ifndef FEAST_ROWS
#define FEAST_ROWS 4
#endif
#ifndef FEAST_MINB
#define FEAST_MINB 3
#endif
static constexpr int kRows = FEAST_ROWS;  // rows per thread gathered in lockstep

__device__ __forceinline__ int find_prob(const FiltProb* probs, int nprob, long long item)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (probs[mid].item0 <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int W>
__device__ __forceinline__ unsigned seg_mask(int sub)
{
    return W == 32 ? 0xffffffffu : (((1u << W) - 1u) << (sub * W));
}

// One CSR row of packed (column, value) entries, read with uniform loads (all
// lanes of a row segment read the same entry, served as one broadcast) and
// gathered against the lane's column of x (and of p when UPD):
//   ax = sum_k a_k x[j_k],  ap = sum_k a_k p[j_k].
// U entries are fetched before any is used, so each warp keeps U (or 2U)
// independent row-segment loads in flight.
template <typename T> __device__ __forceinline__ void load_pk(const void* pk, int t, int& j, T& a);
template <> __device__ __forceinline__ void load_pk<float>(const void* pk, int t, int& j, float& a)
{
    const int2 v = __ldg((const int2*)pk + t);
    j = v.x;
    a = __int_as_float(v.y);
}
template <> __device__ __forceinline__ void load_pk<double>(const void* pk, int t, int& j, double& a)
{
    const int4 v = __ldg((const int4*)pk + t);
    j = v.x;
    a = __hiloint2double(v.w, v.z);
}

template <typename T, int W, bool UPD>
__device__ __forceinline__ void row_gather(const int* __restrict__ ia, const void* __restrict__ pk, int i, int cl,
                                           const c2_t<T>* __restrict__ x, const c2_t<T>* __restrict__ p,
                                           bool use_p, c2_t<T>& ax, c2_t<T>& ap)
{
    using V = c2_t<T>;
    constexpr int U = UPD ? 4 : 8;
    ax = cmk<V>(T(0), T(0));
    ap = cmk<V>(T(0), T(0));
    const int s = __ldg(ia + i), e = __ldg(ia + i + 1);
    for (int t0 = s; t0 < e; t0 += U) {
        V xv[U], pv[U];
        T av[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u;
            int j = 0;
            T aa = T(0);
            if (t < e) load_pk<T>(pk, t, j, aa);
            av[u] = aa;
            xv[u] = (t < e) ? __ldg(x + (size_t)j * W + cl) : cmk<V>(T(0), T(0));
            if (UPD) pv[u] = (t < e && use_p) ? __ldg(p + (size_t)j * W + cl) : cmk<V>(T(0), T(0));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ax.x = fma(av[u], xv[u].x, ax.x);
            ax.y = fma(av[u], xv[u].y, ax.y);
            if (UPD) {
                ap.x = fma(av[u], pv[u].x, ap.x);
                ap.y = fma(av[u], pv[u].y, ap.y);
            }
        }
    }
}

// R rows gathered in lockstep by one thread (rows of the same tile, R*RPP
// apart): the t-th entries of all R rows are fetched together, so the loads
// that miss L2 (the leading edge of a wide stencil) of R rows overlap.
template <typename T, int W, bool UPD, int R>
__device__ __forceinline__ void rows_gather(const int* __restrict__ ia, const void* __restrict__ pk, const int (&row)[R],
                                            int cl, const c2_t<T>* __restrict__ x, const c2_t<T>* __restrict__ p,
                                            bool use_p, c2_t<T> (&ax)[R], c2_t<T> (&ap)[R])
{
    using V = c2_t<T>;
    int s[R], e[R], len = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        s[q] = row[q] >= 0 ? __ldg(ia + row[q]) : 0;
        e[q] = row[q] >= 0 ? __ldg(ia + row[q] + 1) : 0;
        len = max(len, e[q] - s[q]);
        ax[q] = cmk<V>(T(0), T(0));
        ap[q] = cmk<V>(T(0), T(0));
    }
    for (int t = 0; t < len; ++t) {
        V xv[R], pv[R];
        T av[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const bool ok = s[q] + t < e[q];
            int j = 0;
            T aa = T(0);
            if (ok) load_pk<T>(pk, s[q] + t, j, aa);
            av[q] = aa;
            xv[q] = ok ? __ldg(x + (size_t)j * W + cl) : cmk<V>(T(0), T(0));
            if (UPD) pv[q] = (ok && use_p) ? __ldg(p + (size_t)j * W + cl) : cmk<V>(T(0), T(0));
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            ax[q].x = fma(av[q], xv[q].x, ax[q].x);
            ax[q].y = fma(av[q], xv[q].y, ax[q].y);
            if (UPD) {
                ap[q].x = fma(av[q], pv[q].x, ap[q].x);
                ap[q].y = fma(av[q], pv[q].y, ap[q].y);
            }
        }
    }
}

// Block-wide reduction of NV per-thread doubles for each of the W lane
// columns, written to part[item][cl][0..NV).  Fixed order => deterministic.
template <int W, int NV, typename T>
__device__ __forceinline__ void block_partials(T (&v)[NV], double* sm, double* out)
{
    constexpr int SEGS = kThreads / W;
    const int tid = threadIdx.x;
    const int cl = tid % W, seg = tid / W;
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[(seg * W + cl) * NV + q] = (double)v[q];
    __syncthreads();
    if (tid < W) {
        double s[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) s[q] = 0.0;
        for (int g = 0; g < SEGS; ++g)
#pragma unroll
            for (int q = 0; q < NV; ++q) s[q] += sm[(g * W + tid) * NV + q];
#pragma unroll
        for (int q = 0; q < NV; ++q) out[(size_t)tid * kPartStride + q] = s[q];
    }
    __syncthreads();
}

// Called by all threads of the CTA that finished the last item of a group:
// sums the group's partials in item order.  Result in red[cl*kPartStride + q].
template <int W, int NV>
__device__ __forceinline__ void group_reduce(const double* part, long long item_first, int nrb, double* sm,
                                             double* red)
{
    constexpr int SEGS = kThreads / W;
    const int tid = threadIdx.x;
    const int cl = tid % W, seg = tid / W;
    double s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = 0.0;
    for (int rb = seg; rb < nrb; rb += SEGS) {
        const double* src = part + ((size_t)(item_first + rb) * W + cl) * kPartStride;
#pragma unroll
        for (int q = 0; q < NV; ++q) s[q] += __ldcg(src + q);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[(seg * W + cl) * NV + q] = s[q];
    __syncthreads();
    if (tid < W) {
        double t[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) t[q] = 0.0;
        for (int g = 0; g < SEGS; ++g)
#pragma unroll
            for (int q = 0; q < NV; ++q) t[q] += sm[(g * W + tid) * NV + q];
#pragma unroll
        for (int q = 0; q < NV; ++q) red[tid * kPartStride + q] = t[q];
    }
    __syncthreads();
}

// Returns true in every thread of the CTA that completed the group's last item.
__device__ __forceinline__ bool arrive_group(unsigned* counter, int nrb, int* flag_sm)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        *flag_sm = (prev == (unsigned)(nrb - 1));
    }
    __syncthreads();
    const bool last = *flag_sm != 0;
    if (last) __threadfence();
    return last;
}

// ---------------------------------------------------------------- kernel A
template <typename T, int W, bool HASB>
__global__ void __launch_bounds__(kThreads, FEAST_MINB) cocg_step_a(FilterArgs a, int k)
{
    using V = c2_t<T>;
    constexpr int RPP = kThreads / W;  // rows per pass of the CTA
    __shared__ double sm[kThreads * 3];
    __shared__ double red[W * kPartStride];
    __shared__ int flag;
    const int tid = threadIdx.x;
    const int cl = tid % W, sub = (tid % 32) / W, rowslot = tid / W;
    const unsigned mask = seg_mask<W>(sub);
    const bool first = (k == 0);
    const V* pold = (const V*)((k & 1) ? a.p0 : a.p1);
    V* pnew = (V*)((k & 1) ? a.p1 : a.p0);

    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int pi = a.nprob == 1 ? 0 : find_prob(a.probs, a.nprob, item);
        const FiltProb P = a.probs[pi];
        const long long local = item - P.item0;
        const int g = (int)(local / P.nrb), rb = (int)(local % P.nrb);
        if (a.grp_done[P.grp_off + g]) continue;
        ColState* csg = a.cs + P.col_off + (size_t)g * W;
        const int active = csg[cl].active;
        const double2 zd = csg[cl].z, bd = csg[cl].beta;
        const V z = cmk<V>((T)zd.x, (T)zd.y), beta = cmk<V>((T)bd.x, (T)bd.y);
        const bool use_p = !first && active;
        const size_t tile = (size_t)P.vec_off + (size_t)g * P.n * W;
        const V* r = (const V*)a.r + tile;
        const V* po = pold + tile;
        V* pn = pnew + tile;
        T acc[3] = {T(0), T(0), T(0)};  // sigma.re, sigma.im, ||b||^2 (first); FP32 in mixed precision
        const int row0 = rb * a.RB;
        for (int rl = rowslot; rl < a.RB; rl += RPP * kRows) {
            int rows[kRows];
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                const int i = row0 + rl + q * RPP;
                rows[q] = (rl + q * RPP < a.RB && i < P.n) ? i : -1;
            }
            if (rows[0] < 0) break;
            V ar[kRows], ap[kRows];
            rows_gather<T, W, true, kRows>(P.ia, P.apk, rows, cl, r, po, use_p, ar, ap);
            V br[kRows], bp[kRows];
            if (HASB) rows_gather<T, W, true, kRows>(P.ib, P.bpk, rows, cl, r, po, use_p, br, bp);
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                if (rows[q] < 0) continue;
                const int i = rows[q];
                V pi_ = __ldg(r + (size_t)i * W + cl);
                if (use_p) pi_ = cfma(beta, __ldg(po + (size_t)i * W + cl), pi_);
                const V ax = use_p ? cfma(beta, ap[q], ar[q]) : ar[q];  // A (r + beta p)
                V bx = pi_;
                if (HASB) bx = use_p ? cfma(beta, bp[q], br[q]) : br[q];
                const V qv = csub(cmul(z, bx), ax);
                pn[(size_t)i * W + cl] = pi_;
                acc[0] = fma(pi_.x, qv.x, fma(-pi_.y, qv.y, acc[0]));
                acc[1] = fma(pi_.x, qv.y, fma(pi_.y, qv.x, acc[1]));
                if (first) acc[2] = fma(pi_.x, pi_.x, fma(pi_.y, pi_.y, acc[2]));
            }
        }
        block_partials<W, 3>(acc, sm, a.part + (size_t)item * W * kPartStride);
        if (arrive_group(a.grp_count + P.grp_off + g, P.nrb, &flag)) {
            group_reduce<W, 3>(a.part, P.item0 + (long long)g * P.nrb, P.nrb, sm, red);
            if (tid < W) {
                ColState cs = csg[tid];
                if (first) {
                    cs.bn2 = red[tid * kPartStride + 2];
                    cs.rho = make_double2(cs.bn2, 0.0);  // the right-hand side is real
                    cs.rn2 = cs.bn2;
                    if (!(cs.bn2 > 0.0)) { cs.active = 0; cs.status = 1; }
                }
                double2 sig = make_double2(red[tid * kPartStride], red[tid * kPartStride + 1]);
                double2 al = make_double2(0.0, 0.0);
                if (cs.active) {
                    const double d = sig.x * sig.x + sig.y * sig.y;
                    if (!(d > 0.0) || !isfinite(d)) {
                        cs.active = 0;
                        cs.status = 2;
                    } else {  // alpha = rho / sigma
                        al.x = (cs.rho.x * sig.x + cs.rho.y * sig.y) / d;
                        al.y = (cs.rho.y * sig.x - cs.rho.x * sig.y) / d;
                    }
                }
                cs.alpha = al;
                cs.ca = make_double2(cs.c.x * al.x - cs.c.y * al.y, cs.c.x * al.y + cs.c.y * al.x);
                csg[tid] = cs;
            }
            if (tid == 0) a.grp_count[P.grp_off + g] = 0u;
        }
    }
}

// ---------------------------------------------------------------- kernel B
template <typename T, int W, bool HASB>
__global__ void __launch_bounds__(kThreads, FEAST_MINB) cocg_step_b(FilterArgs a, int k)
{
    using V = c2_t<T>;
    constexpr int RPP = kThreads / W;
    __shared__ double sm[kThreads * 3];
    __shared__ double red[W * kPartStride];
    __shared__ int flag;
    const int tid = threadIdx.x;
    const int cl = tid % W, sub = (tid % 32) / W, rowslot = tid / W;
    const unsigned mask = seg_mask<W>(sub);
    const V* pk = (const V*)((k & 1) ? a.p1 : a.p0);
    const int e = cl % a.nbp, mloc = cl / a.nbp;

    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int pi = a.nprob == 1 ? 0 : find_prob(a.probs, a.nprob, item);
        const FiltProb P = a.probs[pi];
        const long long local = item - P.item0;
        const int g = (int)(local / P.nrb), rb = (int)(local % P.nrb);
        if (a.grp_done[P.grp_off + g]) continue;
        ColState* csg = a.cs + P.col_off + (size_t)g * W;
        const int active = csg[cl].active;
        const double2 zd = csg[cl].z, ald = csg[cl].alpha, cad = csg[cl].ca;
        const V z = cmk<V>((T)zd.x, (T)zd.y);
        const V alpha = cmk<V>((T)ald.x, (T)ald.y);
        const V ca = cmk<V>((T)cad.x, (T)cad.y);
        const size_t tile = (size_t)P.vec_off + (size_t)g * P.n * W;
        V* r = (V*)a.r + tile;
        const V* p = pk + tile;
        const int m = g * a.mt + mloc;
        T* dQrow = (T*)a.dQ + P.q_off + m;
        T acc[3] = {T(0), T(0), T(0)};  // rho.re, rho.im, ||r||^2
        const int row0 = rb * a.RB;
        for (int rl = rowslot; rl < a.RB; rl += RPP * kRows) {
            int rows[kRows];
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                const int i = row0 + rl + q * RPP;
                rows[q] = (rl + q * RPP < a.RB && i < P.n) ? i : -1;
            }
            if (rows[0] < 0) break;
            V ax[kRows], unused[kRows], bxs[kRows];
            rows_gather<T, W, false, kRows>(P.ia, P.apk, rows, cl, p, nullptr, false, ax, unused);
            if (HASB) rows_gather<T, W, false, kRows>(P.ib, P.bpk, rows, cl, p, nullptr, false, bxs, unused);
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                const int i = rows[q] < 0 ? 0 : rows[q];
                const bool ok = rows[q] >= 0;
                V pi_ = cmk<V>(T(0), T(0)), ri = cmk<V>(T(0), T(0));
                if (ok) {
                    pi_ = __ldg(p + (size_t)i * W + cl);
                    ri = r[(size_t)i * W + cl];
                }
                const V bx = HASB ? bxs[q] : pi_;
                T qc = T(0);
                if (active && ok) {
                    const V qv = csub(cmul(z, bx), ax[q]);
                    ri = csub(ri, cmul(alpha, qv));
                    r[(size_t)i * W + cl] = ri;
                    qc = ca.x * pi_.x - ca.y * pi_.y;  // Re(c alpha p)
                }
                for (int o = 1; o < a.nbp; o <<= 1) qc += __shfl_xor_sync(mask, qc, o, W);
                if (ok && e == 0 && m < P.m0) dQrow[(size_t)i * P.m0] += qc;
                acc[0] = fma(ri.x, ri.x, fma(-ri.y, ri.y, acc[0]));
                acc[1] = fma(T(2) * ri.x, ri.y, acc[1]);
                acc[2] = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[2]));
            }
        }
        block_partials<W, 3>(acc, sm, a.part + (size_t)item * W * kPartStride);
        if (arrive_group(a.grp_count + P.grp_off + g, P.nrb, &flag)) {
            group_reduce<W, 3>(a.part, P.item0 + (long long)g * P.nrb, P.nrb, sm, red);
            if (tid < 32) {
                int still = 0;
                if (tid < W) {
                    ColState cs = csg[tid];
                    if (cs.active) {
                        const double2 rho1 = make_double2(red[tid * kPartStride], red[tid * kPartStride + 1]);
                        cs.rn2 = red[tid * kPartStride + 2];
                        cs.iters = k + 1;
                        const double d = cs.rho.x * cs.rho.x + cs.rho.y * cs.rho.y;
                        if (cs.rn2 <= a.tol2 * cs.bn2) {
                            cs.active = 0;
                            cs.status = 1;
                        } else if (!(d > 0.0) || !isfinite(cs.rn2)) {
                            cs.active = 0;
                            cs.status = 2;
                        } else {  // beta = rho1 / rho
                            cs.beta.x = (rho1.x * cs.rho.x + rho1.y * cs.rho.y) / d;
                            cs.beta.y = (rho1.y * cs.rho.x - rho1.x * cs.rho.y) / d;
                            cs.rho = rho1;
                        }
                        csg[tid] = cs;
                        still = cs.active;
                    }
                }
                const unsigned anyv = __ballot_sync(0xffffffffu, still);
                if (tid == 0) {
                    if (!anyv) {
                        a.grp_done[P.grp_off + g] = 1;
                        atomicSub(a.groups_left + pi, 1);
                    }
                    if (a.work) atomicAdd(a.work, 1ull);
                    atomicMax(a.iter_max + pi, k + 1);
                    a.grp_count[P.grp_off + g] = 0u;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- init
// Column states for one node batch: node e = node0 + (lane % nbp) of the
// problem's Ne nodes, subspace column m; coefficient c = w_e (first pass) or
// w_e / (z_e - lambda_m) (residual-inverse form); rq = rho(lambda_m) over all
// Ne nodes.  A column is live when m < min(m0, *mk) and e < Ne.
__global__ void colstate_init(const FiltProb* probs, int nprob, ColState* cs, int W, int nbp, int mt,
                              int node0, int rii)
{
    const int pi = blockIdx.y;
    if (pi >= nprob) return;
    const FiltProb P = probs[pi];
    const int ncol = P.G * W;
    const int mk = P.mk ? *P.mk : P.m0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
        const int g = c / W, cl = c % W;
        const int e = node0 + cl % nbp, m = g * mt + cl / nbp;
        ColState s;
        s.rho = s.alpha = s.beta = s.ca = make_double2(0.0, 0.0);
        s.z = s.c = make_double2(0.0, 0.0);
        s.bn2 = s.rn2 = 0.0;
        s.rq = 0.0;
        s.iters = 0;
        s.status = 0;
        s.active = (m < P.m0 && m < mk && e < P.ne) ? 1 : 0;
        if (s.active) {
            const double zr = P.zw[4 * e], zi = P.zw[4 * e + 1], wr = P.zw[4 * e + 2], wi = P.zw[4 * e + 3];
            s.z = make_double2(zr, zi);
            if (rii) {
                const double l = P.lam[m];
                const double dr = zr - l, d2 = dr * dr + zi * zi;
                s.c = make_double2((wr * dr + wi * zi) / d2, (wi * dr - wr * zi) / d2);
                double rq = 0.0;
                for (int f = 0; f < P.ne; ++f) {
                    const double fr = P.zw[4 * f] - l, fi = P.zw[4 * f + 1];
                    rq += (P.zw[4 * f + 2] * fr + P.zw[4 * f + 3] * fi) / (fr * fr + fi * fi);
                }
                s.rq = rq;
            } else {
                s.c = make_double2(wr, wi);
            }
        }
        cs[P.col_off + c] = s;
    }
}

// r <- rhs (real, replicated over the node lanes); with init_q also
// Q <- X diag(rho(lambda)) (residual-inverse form) or Q <- 0 (first pass).
// R and X are the problem's FP64 row-major n x m0 blocks at q_off.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) filter_init(FilterArgs a, const double* R, const double* X,
                                                       int rii, int init_q)
{
    using V = c2_t<T>;
    constexpr int RPP = kThreads / W;
    const int tid = threadIdx.x;
    const int cl = tid % W, rowslot = tid / W;
    const int e = cl % a.nbp, mloc = cl / a.nbp;
    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int pi = a.nprob == 1 ? 0 : find_prob(a.probs, a.nprob, item);
        const FiltProb P = a.probs[pi];
        const long long local = item - P.item0;
        const int g = (int)(local / P.nrb), rb = (int)(local % P.nrb);
        const int m = g * a.mt + mloc;
        const ColState& cs = a.cs[P.col_off + (size_t)g * W + cl];
        const int live = cs.active;
        const double rq = cs.rq;
        const size_t tile = (size_t)P.vec_off + (size_t)g * P.n * W;
        V* r = (V*)a.r + tile;
        const int row0 = rb * a.RB;
        for (int rl = rowslot; rl < a.RB; rl += RPP) {
            const int i = row0 + rl;
            if (i >= P.n) break;
            double v = 0.0;
            if (live) v = R[P.q_off + (size_t)i * P.m0 + m];
            r[(size_t)i * W + cl] = cmk<V>((T)v, T(0));
            if (init_q && e == 0 && m < P.m0) {
                a.Q[P.q_off + (size_t)i * P.m0 + m] = (rii && live) ? rq * X[P.q_off + (size_t)i * P.m0 + m] : 0.0;
                ((T*)a.dQ)[P.q_off + (size_t)i * P.m0 + m] = T(0);
            }
        }
    }
}

// ---------------------------------------------------------------- standalone shifted SpMM
// V = (z B - A) P on the tiled layout (p0 -> r buffer is unused): reads a.p0,
// writes a.p1.  Shifts come from the column states.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) shifted_spmm(FilterArgs a)
{
    using V = c2_t<T>;
    constexpr int RPP = kThreads / W;
    const int tid = threadIdx.x;
    const int cl = tid % W, sub = (tid % 32) / W, rowslot = tid / W;
    const unsigned mask = seg_mask<W>(sub);
    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int pi = a.nprob == 1 ? 0 : find_prob(a.probs, a.nprob, item);
        const FiltProb P = a.probs[pi];
        const long long local = item - P.item0;
        const int g = (int)(local / P.nrb), rb = (int)(local % P.nrb);
        const double2 zd = a.cs[P.col_off + (size_t)g * W + cl].z;
        const V z = cmk<V>((T)zd.x, (T)zd.y);
        const size_t tile = (size_t)P.vec_off + (size_t)g * P.n * W;
        const V* x = (const V*)a.p0 + tile;
        V* y = (V*)a.p1 + tile;
        const int row0 = rb * a.RB;
        for (int rl = rowslot; rl < a.RB; rl += RPP) {
            const int i = row0 + rl;
            if (i >= P.n) break;
            V ax, unused, bx;
            row_gather<T, W, false>(P.ia, P.apk, i, cl, x, nullptr, false, ax, unused);
            if (P.ib == nullptr) bx = __ldg(x + (size_t)i * W + cl);
            else row_gather<T, W, false>(P.ib, P.bpk, i, cl, x, nullptr, false, bx, unused);
            y[(size_t)i * W + cl] = csub(cmul(z, bx), ax);
        }
    }
}

// Q += dQ after all node batches of a pass (dQ: FP32 in mixed precision).
template <typename T>
__global__ void fold_dq(long long total, const T* dQ, double* Q)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        Q[i] += (double)dQ[i];
}

// Packed (column, value) CSR entries for the uniform-load gathers.
__global__ void pack_csr(long long nnz, const int* ja, const double* av, int fp64, void* out)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nnz; t += (long long)gridDim.x * blockDim.x) {
        if (fp64) {
            const double v = av[t];
            ((int4*)out)[t] = make_int4(ja[t], 0, __double2loint(v), __double2hiint(v));
        } else {
            ((int2*)out)[t] = make_int2(ja[t], __float_as_int((float)av[t]));
        }
    }
}

cudaError_t launch_fold_dq(long long total, const void* dQ, bool fp64, double* Q, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > (long long)num_sms() * 8) blocks = (long long)num_sms() * 8;
    if (fp64) fold_dq<double><<<(int)blocks, 256, 0, s>>>(total, (const double*)dQ, Q);
    else fold_dq<float><<<(int)blocks, 256, 0, s>>>(total, (const float*)dQ, Q);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack_csr(long long nnz, const int* ja, const double* av, bool fp64, void* out, cudaStream_t s)
{
    if (nnz <= 0) return cudaSuccess;
    long long blocks = (nnz + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    pack_csr<<<(int)blocks, 256, 0, s>>>(nnz, ja, av, fp64 ? 1 : 0, out);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void cast_values(const double* src, float* dst, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// ---------------------------------------------------------------- dispatch
#define FEAST_DISPATCH(KERNEL, ...)                                                        \
    do {                                                                                   \
        if (fp64) {                                                                        \
            if (a.W == 16) KERNEL<double, 16><<<grid, kThreads, 0, s>>>(__VA_ARGS__);      \
            else if (a.W == 32) KERNEL<double, 32><<<grid, kThreads, 0, s>>>(__VA_ARGS__); \
            else return cudaErrorInvalidValue;                                             \
        } else {                                                                           \
            if (a.W == 16) KERNEL<float, 16><<<grid, kThreads, 0, s>>>(__VA_ARGS__);       \
            else if (a.W == 32) KERNEL<float, 32><<<grid, kThreads, 0, s>>>(__VA_ARGS__);  \
            else return cudaErrorInvalidValue;                                             \
        }                                                                                  \
        count_launches(1);                                                                 \
        return cudaGetLastError();                                                         \
    } while (0)

#define FEAST_DISPATCH_B(KERNEL, ...)                                                      \
    do {                                                                                   \
        if (a.hasB) {                                                                      \
            if (fp64) {                                                                    \
                if (a.W == 16) KERNEL<double, 16, true><<<grid, kThreads, 0, s>>>(__VA_ARGS__);      \
                else if (a.W == 32) KERNEL<double, 32, true><<<grid, kThreads, 0, s>>>(__VA_ARGS__); \
                else return cudaErrorInvalidValue;                                         \
            } else {                                                                       \
                if (a.W == 16) KERNEL<float, 16, true><<<grid, kThreads, 0, s>>>(__VA_ARGS__);       \
                else if (a.W == 32) KERNEL<float, 32, true><<<grid, kThreads, 0, s>>>(__VA_ARGS__);  \
                else return cudaErrorInvalidValue;                                         \
            }                                                                              \
        } else {                                                                           \
            if (fp64) {                                                                    \
                if (a.W == 16) KERNEL<double, 16, false><<<grid, kThreads, 0, s>>>(__VA_ARGS__);      \
                else if (a.W == 32) KERNEL<double, 32, false><<<grid, kThreads, 0, s>>>(__VA_ARGS__); \
                else return cudaErrorInvalidValue;                                         \
            } else {                                                                       \
                if (a.W == 16) KERNEL<float, 16, false><<<grid, kThreads, 0, s>>>(__VA_ARGS__);       \
                else if (a.W == 32) KERNEL<float, 32, false><<<grid, kThreads, 0, s>>>(__VA_ARGS__);  \
                else return cudaErrorInvalidValue;                                         \
            }                                                                              \
        }                                                                                  \
        count_launches(1);                                                                 \
        return cudaGetLastError();                                                         \
    } while (0)

cudaError_t launch_cocg_step_a(const FilterArgs& a, bool fp64, int k, int grid, cudaStream_t s)
{
    FEAST_DISPATCH_B(cocg_step_a, a, k);
}

cudaError_t launch_cocg_step_b(const FilterArgs& a, bool fp64, int k, int grid, cudaStream_t s)
{
    FEAST_DISPATCH_B(cocg_step_b, a, k);
}

cudaError_t launch_filter_init(const FilterArgs& a, bool fp64, const double* R, const double* X, int rii,
                               int init_q, int grid, cudaStream_t s)
{
    FEAST_DISPATCH(filter_init, a, R, X, rii, init_q);
}

cudaError_t launch_colstate_init(const FilterArgs& a, int node0, int rii, cudaStream_t s)
{
    dim3 grid(8, a.nprob);
    colstate_init<<<grid, 256, 0, s>>>(a.probs, a.nprob, a.cs, a.W, a.nbp, a.mt, node0, rii);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_shifted_spmm(const FilterArgs& a, bool fp64, int grid, cudaStream_t s)
{
    FEAST_DISPATCH(shifted_spmm, a);
}

int filter_grid(bool fp64, int W)
{
    int occ = 0;
    cudaError_t e;
    if (fp64) e = W == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cocg_step_b<double, 16, false>, kThreads, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cocg_step_b<double, 32, false>, kThreads, 0);
    else e = W == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cocg_step_b<float, 16, false>, kThreads, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cocg_step_b<float, 32, false>, kThreads, 0);
    if (e != cudaSuccess || occ < 1) occ = 1;
    return num_sms() * occ;
}

cudaError_t launch_cast_values(const double* src, float* dst, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    cast_values<<<(int)blocks, 256, 0, s>>>(src, dst, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace feast
