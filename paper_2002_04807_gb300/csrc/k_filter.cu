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

// Gather sum_k v_k x[j_k] over one CSR row for the lane's column; the row's
// indices and values are loaded once, coalesced, and broadcast by shuffles.
// With UPD, x[j] = r[j] + beta * p[j] is formed on the fly.
template <typename T, int W, bool UPD>
__device__ __forceinline__ c2_t<T> row_gather(const int* __restrict__ ia, const int* __restrict__ ja,
                                              const T* __restrict__ av, int i, unsigned mask, int cl,
                                              const c2_t<T>* __restrict__ x, const c2_t<T>* __restrict__ p,
                                              c2_t<T> beta, bool use_p)
{
    using V = c2_t<T>;
    V acc = cmk<V>(T(0), T(0));
    const int s = __ldg(ia + i), e = __ldg(ia + i + 1);
    for (int base = s; base < e; base += W) {
        const int cnt = min(W, e - base);
        int jl = 0;
        T al = T(0);
        if (cl < cnt) {
            jl = __ldg(ja + base + cl);
            al = __ldg(av + base + cl);
        }
        for (int t = 0; t < cnt; ++t) {
            const int j = __shfl_sync(mask, jl, t, W);
            const T a = __shfl_sync(mask, al, t, W);
            V v = __ldg(x + (size_t)j * W + cl);
            if (UPD && use_p) v = cfma(beta, __ldg(p + (size_t)j * W + cl), v);
            acc.x = fma(a, v.x, acc.x);
            acc.y = fma(a, v.y, acc.y);
        }
    }
    return acc;
}

// Block-wide reduction of NV per-thread doubles for each of the W lane
// columns, written to part[item][cl][0..NV).  Fixed order => deterministic.
template <int W, int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* sm, double* out)
{
    constexpr int SEGS = kThreads / W;
    const int tid = threadIdx.x;
    const int cl = tid % W, seg = tid / W;
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[(seg * W + cl) * NV + q] = v[q];
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
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) cocg_step_a(FilterArgs a, int k)
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
        const T* av = (const T*)P.av;
        const T* bv = (const T*)P.bv;
        double acc[3] = {0.0, 0.0, 0.0};  // sigma.re, sigma.im, ||b||^2 (first)
        const int row0 = rb * a.RB;
        for (int rl = rowslot; rl < a.RB; rl += RPP) {
            const int i = row0 + rl;
            if (i >= P.n) break;
            const V ax = row_gather<T, W, true>(P.ia, P.ja, av, i, mask, cl, r, po, beta, use_p);
            V pi_ = __ldg(r + (size_t)i * W + cl);
            if (use_p) pi_ = cfma(beta, __ldg(po + (size_t)i * W + cl), pi_);
            V bx;
            if (P.ib == nullptr) bx = pi_;
            else bx = row_gather<T, W, true>(P.ib, P.jb, bv, i, mask, cl, r, po, beta, use_p);
            const V q = csub(cmul(z, bx), ax);
            pn[(size_t)i * W + cl] = pi_;
            acc[0] += (double)(pi_.x * q.x - pi_.y * q.y);
            acc[1] += (double)(pi_.x * q.y + pi_.y * q.x);
            if (first) acc[2] += (double)(pi_.x * pi_.x + pi_.y * pi_.y);
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
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) cocg_step_b(FilterArgs a, int k)
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
        const T* av = (const T*)P.av;
        const T* bv = (const T*)P.bv;
        const int m = g * a.mt + mloc;
        double* Qrow = a.Q + P.q_off + m;
        double acc[3] = {0.0, 0.0, 0.0};  // rho.re, rho.im, ||r||^2
        const int row0 = rb * a.RB;
        for (int rl = rowslot; rl < a.RB; rl += RPP) {
            const int i = row0 + rl;
            if (i >= P.n) break;
            const V ax = row_gather<T, W, false>(P.ia, P.ja, av, i, mask, cl, p, nullptr, alpha, false);
            const V pi_ = __ldg(p + (size_t)i * W + cl);
            V bx;
            if (P.ib == nullptr) bx = pi_;
            else bx = row_gather<T, W, false>(P.ib, P.jb, bv, i, mask, cl, p, nullptr, alpha, false);
            V ri = r[(size_t)i * W + cl];
            T qc = T(0);
            if (active) {
                const V q = csub(cmul(z, bx), ax);
                ri = csub(ri, cmul(alpha, q));
                r[(size_t)i * W + cl] = ri;
                qc = ca.x * pi_.x - ca.y * pi_.y;  // Re(c alpha p)
            }
            for (int o = 1; o < a.nbp; o <<= 1) qc += __shfl_xor_sync(mask, qc, o, W);
            if (e == 0 && m < P.m0) Qrow[(size_t)i * P.m0] += (double)qc;
            acc[0] += (double)(ri.x * ri.x - ri.y * ri.y);
            acc[1] += (double)(2 * ri.x * ri.y);
            acc[2] += (double)(ri.x * ri.x + ri.y * ri.y);
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
            if (init_q && e == 0 && m < P.m0)
                a.Q[P.q_off + (size_t)i * P.m0 + m] = (rii && live) ? rq * X[P.q_off + (size_t)i * P.m0 + m] : 0.0;
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
            const V ax = row_gather<T, W, false>(P.ia, P.ja, (const T*)P.av, i, mask, cl, x, nullptr, z, false);
            V bx;
            if (P.ib == nullptr) bx = __ldg(x + (size_t)i * W + cl);
            else bx = row_gather<T, W, false>(P.ib, P.jb, (const T*)P.bv, i, mask, cl, x, nullptr, z, false);
            y[(size_t)i * W + cl] = csub(cmul(z, bx), ax);
        }
    }
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

cudaError_t launch_cocg_step_a(const FilterArgs& a, bool fp64, int k, int grid, cudaStream_t s)
{
    FEAST_DISPATCH(cocg_step_a, a, k);
}

cudaError_t launch_cocg_step_b(const FilterArgs& a, bool fp64, int k, int grid, cudaStream_t s)
{
    FEAST_DISPATCH(cocg_step_b, a, k);
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
    if (fp64) e = W == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cocg_step_b<double, 16>, kThreads, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cocg_step_b<double, 32>, kThreads, 0);
    else e = W == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cocg_step_b<float, 16>, kThreads, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cocg_step_b<float, 32>, kThreads, 0);
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
