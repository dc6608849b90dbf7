// Contour filter kernels: batched complex-shifted CSR SpMM, column-batched
// COCG for the complex symmetric systems (z_e B - A) y = rhs, and the fused
// accumulation of the quadrature sum into the FP64 subspace block Q.
//
// Method (FEAST v4.0 guide, Sec. 1.1 and the tips of Sec. 3.1): for the Ne
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
//   A: s = (zB - A) r_k (the only gather), p_k = r_k + beta p_{k-1} and
//      q_k = s + beta q_{k-1} = (zB - A) p_k in place, partial sums of
//      p_k^T q_k; the last item of a group sets alpha = rho / p^T q.
//   B: streaming only: r -= alpha q, Q += Re(c alpha p_k), partial sums of
//      r^T r and |r|^2; the last item sets beta and each column's state.
// Carrying q by its recurrence means one gathered vector per step: on GB300
// a gather of a wide 3D stencil moves data at roughly half the rate of a
// plain stream (far neighbours come through L2), so trading a second gather
// for two extra streams is faster even though it moves more bytes.
// Step A comes in three forms: the gather through the caches (cocg_step_a,
// any matrix, several problems), and for single problems whose row blocks
// read a few contiguous column ranges the staged forms, which copy those
// ranges of r into shared memory with bulk asynchronous copies first: two
// CTAs per SM each loading then computing one item (cocg_step_aw), or one
// CTA per SM with a producer warp filling two stages while 16 warps compute
// (cocg_step_ws, for blocks that stage many rows per row).
// Rows of a CSR matrix are stored as packed (column, value) entries, the
// diagonal entry first, padded to chunks of 8 with column -1 entries that
// issue no load, so a row is gathered with fully unrolled loads and its own
// value comes out of its first load.
// Reductions are deterministic: fixed per-thread order, fixed block order;
// every work item (staged forms: every CTA, once per group) writes its own
// partial-sum slot, the CTA that completes a bucket of 32 consecutive slots
// sums them into a bucket slot, and the CTA that completes a group's last
// bucket sums the bucket slots, each in slot order.  No CTA has to read more
// than 64 slots, so no single CTA carries a long reduction at the end of a
// launch.  Per-thread and per-item sums run in the filter precision: GB300's
// FP64 rate is a small fraction of its FP32 rate.
#include "feast_internal.cuh"
#include <climits>
#include <algorithm>

namespace feast {

static constexpr int kThreads = 256;
static constexpr int kPartStride = 4;
static constexpr int kChunk = 8;  // padded CSR chunk (entries)
// Packed entries of one item staged in shared memory.  Kept small: shared
// memory comes out of the L1 capacity that caches the gathered neighbours.
static constexpr int kStageEntries = 2048;
static constexpr int kMaxRB = 512;  // rows per work item, at most
#ifndef FEAST_MINB
#define FEAST_MINB 5
#endif
#ifndef FEAST_MINB_B
#define FEAST_MINB_B 4
#endif
#ifndef FEAST_AW_MINB
#define FEAST_AW_MINB 2  // resident CTAs per SM the staged step A is compiled for
#endif
#ifndef FEAST_B_ROWS
#define FEAST_B_ROWS 4  // streaming step: rows per thread whose loads are issued together
#endif

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

// ---------------------------------------------------------------- padded CSR chunks
// Entries of a packed row chunk: float entries are 8 bytes (two per int4),
// double entries 16 bytes (one per int4).  SH: the entries sit in shared
// memory (plain loads) rather than global memory (read-only cache loads).
template <typename T, bool SH> __device__ __forceinline__ void load_chunk(const int4* ent, int c, int (&j)[kChunk], T (&a)[kChunk]);
template <> __device__ __forceinline__ void load_chunk<float, true>(const int4* ent, int c, int (&j)[kChunk], float (&a)[kChunk])
{
    const int4* q = ent + (c >> 1);
#pragma unroll
    for (int u = 0; u < kChunk / 2; ++u) {
        const int4 v = q[u];
        j[2 * u] = v.x;
        a[2 * u] = __int_as_float(v.y);
        j[2 * u + 1] = v.z;
        a[2 * u + 1] = __int_as_float(v.w);
    }
}
template <> __device__ __forceinline__ void load_chunk<float, false>(const int4* ent, int c, int (&j)[kChunk], float (&a)[kChunk])
{
    const int4* q = ent + (c >> 1);
#pragma unroll
    for (int u = 0; u < kChunk / 2; ++u) {
        const int4 v = __ldg(q + u);
        j[2 * u] = v.x;
        a[2 * u] = __int_as_float(v.y);
        j[2 * u + 1] = v.z;
        a[2 * u + 1] = __int_as_float(v.w);
    }
}
template <> __device__ __forceinline__ void load_chunk<double, true>(const int4* ent, int c, int (&j)[kChunk], double (&a)[kChunk])
{
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
        const int4 v = ent[c + u];
        j[u] = v.x;
        a[u] = __hiloint2double(v.w, v.z);
    }
}
template <> __device__ __forceinline__ void load_chunk<double, false>(const int4* ent, int c, int (&j)[kChunk], double (&a)[kChunk])
{
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
        const int4 v = __ldg(ent + c + u);
        j[u] = v.x;
        a[u] = __hiloint2double(v.w, v.z);
    }
}

// ax = sum a_k x[j_k] over the padded row entries [c0, c1) of ent (padding
// entries have column -1 and issue no load).  The row's own value x[i] comes
// out of the same loads when the row stores column i; *own says whether it did.
template <typename T, int W, bool SH>
__device__ __forceinline__ void row_gather(const int4* __restrict__ ent, int c0, int c1, int i,
                                           const c2_t<T>* __restrict__ xl, c2_t<T>& ax, c2_t<T>& xo, bool& own)
{
    using V = c2_t<T>;
    ax = cmk<V>(T(0), T(0));
    own = false;
    for (int c = c0; c < c1; c += kChunk) {
        int j[kChunk];
        T av[kChunk];
        load_chunk<T, SH>(ent, c, j, av);
        V xv[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) xv[u] = j[u] >= 0 ? __ldg(xl + (size_t)j[u] * W) : cmk<V>(T(0), T(0));
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
            ax.x = fma(av[u], xv[u].x, ax.x);
            ax.y = fma(av[u], xv[u].y, ax.y);
            if (j[u] == i) {
                xo = xv[u];
                own = true;
            }
        }
    }
}

// Row gather that reads the entries from global memory (rows of B, and the
// standalone SpMM).
template <typename T, int W>
__device__ __forceinline__ c2_t<T> row_gather_global(const int* __restrict__ pp, const void* __restrict__ pk, int i,
                                                     const c2_t<T>* __restrict__ xl)
{
    c2_t<T> ax, xo;
    bool own;
    row_gather<T, W, false>((const int4*)pk, __ldg(pp + i), __ldg(pp + i + 1), i, xl, ax, xo, own);
    return ax;
}

// Stage the packed entries of rows [row0, row1) in shared memory (one
// coalesced copy per item) together with their row offsets.  Returns the
// entries' base (shared when they fit, else global) and whether staged.
template <typename T>
__device__ __forceinline__ bool stage_rows(const int* __restrict__ pp, const void* __restrict__ pk, int row0, int row1,
                                           int* s_pp, int4* s_ent, const int4*& gent)
{
    constexpr int EPI = sizeof(T) == 4 ? 2 : 1;  // entries per int4
    const int rows = row1 - row0;
    const int c_lo = __ldg(pp + row0);
    for (int t = threadIdx.x; t <= rows; t += kThreads) s_pp[t] = __ldg(pp + row0 + t) - c_lo;
    __syncthreads();
    const int cnt = s_pp[rows];
    gent = (const int4*)pk + c_lo / EPI;
    const bool staged = cnt <= kStageEntries;
    if (staged)
        for (int t = threadIdx.x; t < cnt / EPI; t += kThreads) s_ent[t] = __ldg(gent + t);
    __syncthreads();
    return staged;
}

// ---------------------------------------------------------------- reductions
// Barrier policies: the whole CTA, or the NT threads of named barrier ID (the
// consumer warps of a warp-specialized kernel, whose producer warp does not
// take part).
struct CtaSync {
    static __device__ __forceinline__ void sync() { __syncthreads(); }
};
template <int ID, int NT>
struct NamedSync {
    static __device__ __forceinline__ void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NT) : "memory"); }
};

// Block-wide reduction of NV per-thread values for each of the W lane columns,
// written to the work item's slot.  A slot holds kPartStride rows of W
// doubles (slot[q * W + cl]), so one value of every lane is one coalesced
// row.  Fixed order.
// The sums run in the values' own type and only the W results are widened:
// GB300 issues FP64 arithmetic and conversions at a small fraction of the FP32
// rate, so per-thread FP64 work in a per-item reduction costs more than the item.
template <int W, int NV, typename T, int NT = kThreads, typename SY = CtaSync>
__device__ __forceinline__ void item_partials(T (&v)[NV], double* sm, double* slot)
{
    constexpr int SEGS = NT / W;
    const int tid = threadIdx.x;
    const int cl = tid % W, seg = tid / W;
    T* st = reinterpret_cast<T*>(sm);
#pragma unroll
    for (int q = 0; q < NV; ++q) st[(seg * W + cl) * NV + q] = v[q];
    SY::sync();
    if (tid < W) {
        T s[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) s[q] = T(0);
        for (int g = 0; g < SEGS; ++g)
#pragma unroll
            for (int q = 0; q < NV; ++q) s[q] += st[(g * W + tid) * NV + q];
#pragma unroll
        for (int q = 0; q < NV; ++q) slot[(size_t)q * W + tid] = (double)s[q];
    }
    SY::sync();
}

// Compensated (Kahan) running sum in the filter precision: s - c carries the
// sum of the added values to about one rounding of the type.
template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x)
{
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

// Sum of `count` consecutive slots starting at `base`, per lane, in a fixed
// order, into red[cl * kPartStride + q] (shared).  All threads of the CTA.
template <int W, int NV, int NT = kThreads, typename SY = CtaSync>
__device__ __forceinline__ void sum_slots(const double* base, int count, double* sm, double* red)
{
    constexpr int SEGS = NT / W;
    const int tid = threadIdx.x;
    const int cl = tid % W, seg = tid / W;
    double s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = 0.0;
#pragma unroll 4
    for (int b = seg; b < count; b += SEGS)
#pragma unroll
        for (int q = 0; q < NV; ++q) s[q] += __ldcg(base + ((size_t)b * kPartStride + q) * W + cl);
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[(seg * W + cl) * NV + q] = s[q];
    SY::sync();
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
    SY::sync();
}

// Returns true in every thread of the CTA whose arrival is the total-th.
template <typename SY = CtaSync>
__device__ __forceinline__ bool arrive_count(unsigned* counter, int total, int* flag_sm)
{
    __threadfence();
    SY::sync();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        *flag_sm = (prev == (unsigned)(total - 1));
    }
    SY::sync();
    const bool last = *flag_sm != 0;
    if (last) __threadfence();
    return last;
}

// After an item wrote its slot: the CTA completing the item's bucket sums the
// bucket into its bucket slot; the CTA completing the group's last bucket sums
// the bucket slots into red[] and returns true (all its threads).  Counters
// are reset by the CTA that completes them.
template <int W, int NV, int NT = kThreads, typename SY = CtaSync>
__device__ __forceinline__ bool tree_arrive(double* gslots, int nrb, int rb, unsigned* bk_count, unsigned* grp_count,
                                            double* sm, double* red, int* flag_sm)
{
    const int nbk = part_buckets(nrb);
    const int bk = rb / kPartBucket;
    const int bsz = min(kPartBucket, nrb - bk * kPartBucket);
    if (!arrive_count<SY>(bk_count + bk, bsz, flag_sm)) return false;
    sum_slots<W, NV, NT, SY>(gslots + (size_t)bk * kPartBucket * kPartStride * W, bsz, sm, red);
    if (threadIdx.x < W) {
        double* bs = gslots + ((size_t)nrb + bk) * kPartStride * W;
#pragma unroll
        for (int q = 0; q < NV; ++q) bs[(size_t)q * W + threadIdx.x] = red[threadIdx.x * kPartStride + q];
    }
    if (threadIdx.x == 0) bk_count[bk] = 0u;
    if (!arrive_count<SY>(grp_count, nbk, flag_sm)) return false;
    sum_slots<W, NV, NT, SY>(gslots + (size_t)nrb * kPartStride * W, nbk, sm, red);
    if (threadIdx.x == 0) *grp_count = 0u;
    return true;
}

struct ItemInfo {
    int pi, g, rb;
};

__device__ __forceinline__ ItemInfo item_info(const FilterArgs& a, long long item)
{
    ItemInfo t;
    t.pi = a.nprob == 1 ? 0 : (a.item_prob ? a.item_prob[item] : find_prob(a.probs, a.nprob, item));
    const long long local = item - a.probs[t.pi].item0;
    const int nrb = a.probs[t.pi].nrb;
    t.g = (int)(local / nrb);
    t.rb = (int)(local % nrb);
    return t;
}

// Items of the streaming step use their own, larger row blocks (RBb rows).
__device__ __forceinline__ int find_prob_b(const FiltProb* probs, int nprob, long long item)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (probs[mid].item0_b <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ ItemInfo item_info_b(const FilterArgs& a, long long item)
{
    ItemInfo t;
    t.pi = a.nprob == 1 ? 0 : (a.item_prob_b ? a.item_prob_b[item] : find_prob_b(a.probs, a.nprob, item));
    const long long local = item - a.probs[t.pi].item0_b;
    const int nrb = a.probs[t.pi].nrb_b;
    t.g = (int)(local / nrb);
    t.rb = (int)(local % nrb);
    return t;
}

// ---------------------------------------------------------------- group finish
// Run by the CTA that completed a group's last item.  Kept out of line so
// that their FP64 scalar work does not raise the register count of the
// streaming loops.  Step A: sigma = p^T q, alpha = rho / sigma, c alpha.
template <int W>
__device__ __noinline__ void finish_group_a(ColState* csg, bool first, const double* red)
{
    const int tid = threadIdx.x;
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
}

// Step B: rho' = r^T r, beta = rho' / rho, convergence |r|^2 <= tol^2 |b|^2;
// a group whose columns all stopped is marked done.
template <int W>
__device__ __noinline__ void finish_group_b(ColState* csg, int k, double tol2, int* done, int* groups_left,
                                            int* iter_max, unsigned long long* work, const double* red)
{
    const int tid = threadIdx.x;
    if (tid < 32) {
        int still = 0;
        if (tid < W) {
            ColState cs = csg[tid];
            if (cs.active) {
                const double2 rho1 = make_double2(red[tid * kPartStride], red[tid * kPartStride + 1]);
                cs.rn2 = red[tid * kPartStride + 2];
                cs.iters = k + 1;
                const double d = cs.rho.x * cs.rho.x + cs.rho.y * cs.rho.y;
                if (cs.rn2 <= tol2 * cs.bn2) {
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
                *done = 1;
                atomicSub(groups_left, 1);
            }
            if (work) atomicAdd(work, 1ull);
            atomicMax(iter_max, k + 1);
        }
    }
}

// ---------------------------------------------------------------- kernel A
// s = (zB - A) r_k gathered over the matrix rows; then, per own row,
// p_k = r_k + beta_k p_{k-1}, q_k = s + beta_k q_{k-1} (= (zB - A) p_k),
// both updated in place, and partial sums of p_k^T q_k (and ||r_0||^2 at k=0).
// BM: 0 = B is the identity, 1 = B diagonal (values bd), 2 = general CSR B.
template <typename T, int W, int BM>
__global__ void __launch_bounds__(kThreads, FEAST_MINB) cocg_step_a(FilterArgs a, int kk)
{
    const int k = a.kdev ? *a.kdev : kk;  // step index (read from the device when replayed in a graph)
    using V = c2_t<T>;
    constexpr int RPP = kThreads / W;  // rows per pass of the CTA
    constexpr int STAGE4 = sizeof(T) == 4 ? kStageEntries / 2 : kStageEntries;
    __shared__ double sm[kThreads * 3];
    __shared__ double red[W * kPartStride];
    __shared__ int flag;
    __shared__ int s_pp[kMaxRB + 1];
    __shared__ int4 s_ent[STAGE4];
    const int tid = threadIdx.x;
    const int cl = tid % W, rowslot = tid / W;
    const bool first = (k == 0);

    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const ItemInfo it = item_info(a, item);
        const FiltProb& P = a.probs[it.pi];
        const int g = it.g;
        if (a.grp_done[P.grp_off + g]) continue;
        ColState* csg = a.cs + P.col_off + (size_t)g * W;
        const int active = csg[cl].active;
        const double2 zd = csg[cl].z, bd = csg[cl].beta;
        const V z = cmk<V>((T)zd.x, (T)zd.y), beta = cmk<V>((T)bd.x, (T)bd.y);
        const bool use_p = !first && active;
        const int n = P.n;
        const size_t tile = (size_t)P.vec_off + (size_t)g * n * W;
        const V* rl_ = (const V*)a.r + tile + cl;
        V* pl_ = (V*)a.p0 + tile + cl;
        V* ql_ = (V*)a.p1 + tile + cl;
        T acc[3] = {T(0), T(0), T(0)};  // sigma.re, sigma.im, ||b||^2 (first)
        const int row0 = it.rb * a.RB;
        const int row1 = min(n, row0 + a.RB);
        const int4* gent;
        const bool staged = stage_rows<T>(P.app, P.apk, row0, row1, s_pp, s_ent, gent);
        const V zero = cmk<V>(T(0), T(0));
        for (int i = row0 + rowslot; i < row1; i += RPP) {
            // own-row streams first, so their loads overlap the gather
            V po = zero, qo = zero;
            if (use_p) {
                po = pl_[(size_t)i * W];
                qo = ql_[(size_t)i * W];
            }
            const int c0 = s_pp[i - row0], c1 = s_pp[i - row0 + 1];
            V ar, ri = zero;
            bool own;
            if (staged) row_gather<T, W, true>(s_ent, c0, c1, i, rl_, ar, ri, own);
            else row_gather<T, W, false>(gent, c0, c1, i, rl_, ar, ri, own);
            if (!own) ri = __ldg(rl_ + (size_t)i * W);
            V bx = ri;
            if (BM == 1) {
                const T b = ((const T*)P.bd)[i];
                bx = cmk<V>(b * ri.x, b * ri.y);
            } else if (BM == 2) {
                bx = row_gather_global<T, W>(P.bpp, P.bpk, i, rl_);
            }
            V pi_ = ri, qi = csub(cmul(z, bx), ar);  // (zB - A) r
            if (use_p) {
                pi_ = cfma(beta, po, pi_);
                qi = cfma(beta, qo, qi);
            }
            pl_[(size_t)i * W] = pi_;
            ql_[(size_t)i * W] = qi;
            acc[0] = fma(pi_.x, qi.x, fma(-pi_.y, qi.y, acc[0]));
            acc[1] = fma(pi_.x, qi.y, fma(pi_.y, qi.x, acc[1]));
            if (first) acc[2] = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[2]));
        }
        const int gi = P.grp_off + g;
        double* gslots = a.part + (size_t)gi * a.nslot * kPartStride * W;
        item_partials<W, 3>(acc, sm, gslots + (size_t)it.rb * kPartStride * W);
        if (tree_arrive<W, 3>(gslots, P.nrb, it.rb, a.bk_count + (size_t)gi * a.nbk, a.grp_count + gi, sm, red, &flag))
            finish_group_a<W>(csg, first, red);
    }
}

// ---------------------------------------------------------------- kernel B
// Pure streaming over own rows: r_{k+1} = r_k - alpha q_k, the quadrature
// accumulator += Re(c alpha p_k) (summed over the node lanes of a column),
// partial sums of r^T r and |r|^2; the last item of a group sets beta and
// the columns' convergence state.
template <typename T, int W, int BM>
__global__ void __launch_bounds__(kThreads, FEAST_MINB_B) cocg_step_b(FilterArgs a, int kk)
{
    const int k = a.kdev ? *a.kdev : kk;
    using V = c2_t<T>;
    constexpr int RPP = kThreads / W;
    __shared__ double sm[kThreads * 3];
    __shared__ double red[W * kPartStride];
    __shared__ int flag;
    const int tid = threadIdx.x;
    const int cl = tid % W, sub = (tid % 32) / W, rowslot = tid / W;
    const unsigned mask = seg_mask<W>(sub);
    const int e = cl % a.nbp, mloc = cl / a.nbp;

    for (long long item = blockIdx.x; item < a.nitems_b; item += gridDim.x) {
        const ItemInfo it = item_info_b(a, item);
        const FiltProb& P = a.probs[it.pi];
        const int g = it.g;
        if (a.grp_done[P.grp_off + g]) continue;
        ColState* csg = a.cs + P.col_off + (size_t)g * W;
        const int active = csg[cl].active;
        const double2 ald = csg[cl].alpha, cad = csg[cl].ca;
        const V alpha = cmk<V>((T)ald.x, (T)ald.y);
        const V ca = cmk<V>((T)cad.x, (T)cad.y);
        const int n = P.n;
        const size_t tile = (size_t)P.vec_off + (size_t)g * n * W;
        V* r = (V*)a.r + tile + cl;
        const V* pl_ = (const V*)a.p0 + tile + cl;
        const V* ql_ = (const V*)a.p1 + tile + cl;
        const int m = g * a.mt + mloc;
        T* dQt = (T*)a.dQ + P.dq_off + (size_t)g * n * a.mt + mloc;  // [group][row][mt] tile
        const bool writes_q = (e == 0 && m < P.m0);
        T acc[3] = {T(0), T(0), T(0)};  // rho.re, rho.im, ||r||^2
        const int row0 = it.rb * a.RBb;
        const int row1 = min(n, row0 + a.RBb);
        // FEAST_B_ROWS rows per thread per pass, every load issued before any use
        constexpr int U = FEAST_B_ROWS;
        for (int i0 = row0 + rowslot; i0 < row1; i0 += U * RPP) {
            int ii[U];
#pragma unroll
            for (int u = 0; u < U; ++u) ii[u] = i0 + u * RPP;
            V rv[U], pv[U], qv[U];
            T dq[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = ii[u] < row1;
                const size_t o = (size_t)(ok ? ii[u] : i0) * W;
                rv[u] = ok ? r[o] : cmk<V>(T(0), T(0));
                pv[u] = (ok && active) ? __ldg(pl_ + o) : cmk<V>(T(0), T(0));
                qv[u] = (ok && active) ? __ldg(ql_ + o) : cmk<V>(T(0), T(0));
                dq[u] = (ok && writes_q) ? dQt[(size_t)(ok ? ii[u] : i0) * a.mt] : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = ii[u] < row1;
                V ri = rv[u];
                T qc = T(0);
                if (active) {
                    ri = csub(ri, cmul(alpha, qv[u]));
                    if (ok) r[(size_t)ii[u] * W] = ri;
                    qc = ca.x * pv[u].x - ca.y * pv[u].y;  // Re(c alpha p)
                }
                for (int o = 1; o < a.nbp; o <<= 1) qc += __shfl_xor_sync(mask, qc, o, W);
                if (ok && writes_q) dQt[(size_t)ii[u] * a.mt] = dq[u] + qc;
                acc[0] = fma(ri.x, ri.x, fma(-ri.y, ri.y, acc[0]));
                acc[1] = fma(T(2) * ri.x, ri.y, acc[1]);
                acc[2] = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[2]));
            }
        }
        const int gi = P.grp_off + g;
        double* gslots = a.part + (size_t)gi * a.nslot * kPartStride * W;
        item_partials<W, 3>(acc, sm, gslots + (size_t)it.rb * kPartStride * W);
        if (tree_arrive<W, 3>(gslots, P.nrb_b, it.rb, a.bk_count + (size_t)gi * a.nbk, a.grp_count + gi, sm, red,
                              &flag))
            finish_group_b<W>(csg, k, a.tol2, a.grp_done + gi, a.groups_left + it.pi, a.iter_max + it.pi, a.work, red);
    }
}

// ---------------------------------------------------------------- staged-window gather
// Step A's rows read r at the columns of their entries.  For matrices whose
// row blocks touch a few contiguous column ranges (stencils and other
// locally numbered problems), a work item of RBW rows copies exactly those
// ranges ("windows") of the group tile into shared memory with bulk
// asynchronous copies -- one instruction per window, no registers held while
// the bytes are in flight -- and gathers from shared memory.  The entries'
// column indices are rewritten once per matrix into positions within the row
// block's staged windows (win_build).  A CTA accumulates its partial sums over
// all its items of a group and publishes them once per group, so the
// publication cost (a fence and a counter) is paid per CTA, not per item.
static constexpr int kWinGap = 4;      // column gaps up to this many rows are staged rather than split
static constexpr int kWinKeys = 4096;  // sort capacity per row block (entries + own rows)

__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned addr, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity: false after `limit` SM
// clock cycles without completion.
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity, long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try(addr, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// Limit of the wait for copies still in flight after a timed-out wait, before a
// CTA leaves: at least about a second, whatever the caller's limit, so that no
// copy lands in shared memory after its CTA has exited.
__device__ __forceinline__ long long settle_limit(long long limit) { return limit > 2000000000LL ? limit : 2000000000LL; }

// Bulk copy global -> shared (TMA engine), completion counted on the mbarrier.
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Ascending bitonic sort of key[0, P2) in shared memory (P2 a power of two);
// all threads of the CTA take part.
__device__ void block_bitonic(int* key, int P2)
{
    for (int k = 2; k <= P2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P2; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const int a = key[t], b = key[u];
                    if ((a > b) == ((t & k) == 0)) {
                        key[t] = b;
                        key[u] = a;
                    }
                }
            }
            __syncthreads();
        }
}

// One CTA per row block (grid-stride): the distinct columns of its entries
// and its own rows, sorted and merged into windows; entries rewritten with
// staged positions (window base + column - window start).
// Each row block's staged metadata is one contiguous region of `meta`, at
// byte offset rb * (rbw + 4) * 4 + e0 * sizeof(PK) (e0: the block's first
// packed entry), so one bulk copy stages it: (rbw + 4) ints -- the row
// pointers relative to e0 (t = 0..rbw; rows past the end repeat the last), the
// own rows' staged position at t = rbw + 1 -- then the block's entries with
// staged positions for columns.
template <typename PK>
__global__ void __launch_bounds__(256) win_build(int n, int rbw, int nrbw, const int* __restrict__ pp,
                                                 const PK* __restrict__ pk, char* __restrict__ meta,
                                                 int4* __restrict__ hdr, int2* __restrict__ win, int* stat)
{
    __shared__ int key[kWinKeys];
    __shared__ int ws[kWinMax], we[kWinMax], wb[kWinMax];
    __shared__ int s_kv, s_nw, s_ok;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int rb = blockIdx.x; rb < nrbw; rb += gridDim.x) {
        const int row0 = rb * rbw, row1 = min(n, row0 + rbw), rows = row1 - row0;
        const int e0 = pp[row0], cnt = pp[row1] - e0;
        const int K = cnt + rows;
        if (K > kWinKeys) {
            if (tid == 0) atomicAdd(stat + 2, 1);
            continue;
        }
        int P2 = 1;
        while (P2 < K) P2 <<= 1;
        int bad = 0;
        for (int t = tid; t < P2; t += blockDim.x) {
            int kv = INT_MAX;
            if (t < cnt) {
                const int j = pk[e0 + t].x;
                if (j < -1 || j >= n) bad = 1;
                else if (j >= 0) kv = j;
            } else if (t < K) {
                kv = row0 + (t - cnt);
            }
            key[t] = kv;
        }
        if (tid == 0) s_kv = 0;
        if (__syncthreads_or(bad)) {
            if (tid == 0) atomicAdd(stat + 3, 1);
            continue;
        }
        block_bitonic(key, P2);
        for (int t = tid; t < P2; t += blockDim.x)
            if (key[t] != INT_MAX && (t + 1 == P2 || key[t + 1] == INT_MAX)) s_kv = t + 1;
        __syncthreads();
        if (tid < 32) {  // windows: runs of keys with gaps <= kWinGap
            const int kv = s_kv;
            int nw = 0;
            for (int base = 0; base < kv; base += 32) {
                const int t = base + lane;
                const int k = t < kv ? key[t] : 0;
                const bool st = t < kv && (t == 0 || k - key[t - 1] > kWinGap);
                const bool en = t < kv && (t + 1 == kv || key[t + 1] - k > kWinGap);
                const unsigned m = __ballot_sync(0xffffffffu, st);
                if (st) {
                    const int w = nw + __popc(m & ((1u << lane) - 1u));
                    if (w < kWinMax) ws[w] = k;
                }
                if (en) {
                    const int w = nw + __popc(m & ((2u << lane) - 1u)) - 1;
                    if (w < kWinMax) we[w] = k + 1;
                }
                nw += __popc(m);
            }
            __syncwarp();
            if (lane == 0) {
                int ok = nw <= kWinMax, total = 0, own = 0;
                if (ok) {
                    for (int w = 0; w < nw; ++w) {
                        wb[w] = total;
                        if (ws[w] <= row0 && row0 < we[w]) own = total + row0 - ws[w];
                        win[(size_t)rb * kWinMax + w] = make_int2(ws[w], we[w] - ws[w]);
                        total += we[w] - ws[w];
                    }
                    hdr[rb] = make_int4(nw, total, own, cnt);
                    int* lpp = (int*)(meta + (size_t)rb * (rbw + 4) * 4 + (size_t)e0 * sizeof(PK));
                    lpp[rbw + 1] = own;
                    lpp[rbw + 2] = 0;
                    lpp[rbw + 3] = 0;
                    atomicMax(stat + 0, total);
                    atomicMax(stat + 1, cnt);
                } else {
                    atomicAdd(stat + 2, 1);
                }
                s_nw = nw;
                s_ok = ok;
            }
        }
        __syncthreads();
        if (s_ok) {
            const int nw = s_nw;
            char* region = meta + (size_t)rb * (rbw + 4) * 4 + (size_t)e0 * sizeof(PK);
            int* lpp = (int*)region;
            PK* lpk = (PK*)(region + (size_t)(rbw + 4) * 4);
            for (int t = tid; t <= rbw; t += blockDim.x) lpp[t] = pp[min(row0 + t, row1)] - e0;
            for (int t = tid; t < cnt; t += blockDim.x) {
                PK e = pk[e0 + t];
                if (e.x >= 0) {
                    int w = 0;
                    while (w + 1 < nw && e.x >= ws[w + 1]) ++w;
                    e.x = wb[w] + e.x - ws[w];
                }
                lpk[t] = e;
            }
        }
        __syncthreads();  // shared tables are rewritten by the next row block
    }
}

// Step A on staged windows: same arithmetic as cocg_step_a (s = (zB - A) r,
// p = r + beta p, q = s + beta q, partial sums of p^T q and, at k = 0,
// ||r||^2), single problem, B the identity (BM 0) or diagonal (BM 1).  The
// launch grid must not exceed the row blocks per group, so that every CTA
// has items in every group and each group's partial sums arrive from exactly
// gridDim.x CTAs (slot = blockIdx.x).  Work items are counted in 32-bit ints
// (checked by the host).
template <typename T, int W, int BM, int RBW>
__global__ void __launch_bounds__(kThreads, FEAST_AW_MINB) cocg_step_aw(FilterArgs a, int kk)
{
    const int k = a.kdev ? *a.kdev : kk;
    using V = c2_t<T>;
    constexpr int RPP = kThreads / W;   // rows per pass of the CTA
    constexpr int RPT = RBW / RPP;      // rows per thread per item
    static_assert(RBW % RPP == 0, "row block must be a whole number of passes");
    constexpr int LPP = RBW + 4;        // local row pointers + own position, per row block
    constexpr unsigned ROWB = W * sizeof(V);                // bytes per tile row
    constexpr unsigned ENTB = sizeof(T) == 4 ? 8u : 16u;    // bytes per packed entry
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ double sm[kThreads * 3];
    __shared__ double red[W * kPartStride];
    __shared__ int flag;
    __shared__ __align__(8) unsigned long long mbar;
    const int tid = threadIdx.x, lane = tid & 31;
    const int cl = tid % W, rowslot = tid / W;
    const bool first = (k == 0);
    // dynamic shared memory from a 128-byte boundary (bulk copies need 16-byte
    // aligned destinations; the request includes the pad): staged rows, the
    // row block's entries, its local row pointers
    const unsigned dsm_sh = (unsigned)__cvta_generic_to_shared(dsm);
    const unsigned xs_sh = (dsm_sh + 127u) & ~127u;
    const unsigned lpp_sh = xs_sh + (unsigned)a.wcapr * ROWB;  // staged metadata: row pointers, then entries
    const unsigned ent_sh = lpp_sh + LPP * 4u;
    const V* xs = (const V*)(dsm + (xs_sh - dsm_sh));
    const int4* sent = (const int4*)(dsm + (ent_sh - dsm_sh));
    const int* lp = (const int*)(dsm + (lpp_sh - dsm_sh));
    const unsigned mb = (unsigned)__cvta_generic_to_shared(&mbar);
    if (tid == 0) {
        mbar_init(mb, 1);
        mbar_fence_init();
    }
    __syncthreads();
    unsigned parity = 0;

    const FiltProb& P = a.probs[0];
    const int n = P.n, nrb = P.nrb, nitems = (int)a.nitems;
    const int* __restrict__ app = P.app;
    const V zero = cmk<V>(T(0), T(0));
    int cur = -1;
    bool skip = false, use_p = false;
    V z = zero, beta = zero;
    V *pl_ = nullptr, *ql_ = nullptr;
    const char* rtile = nullptr;
    T accs[3] = {T(0), T(0), T(0)}, accc[3] = {T(0), T(0), T(0)};  // this CTA's run sums (compensated)
    int4 mh = make_int4(0, 0, 0, 0);  // warp 0: table rows of row block mrb
    int2 mwv = make_int2(0, 0);
    int me0 = 0, mrb = -1;
    for (int item = blockIdx.x;; item += gridDim.x) {
        const bool have = item < nitems;
        const int g = have ? item / nrb : -1;
        if (g != cur) {
            if (cur >= 0 && !skip) {  // publish this CTA's sums over its items of group cur
                const int gi = P.grp_off + cur;
                double* gslots = a.part + (size_t)gi * a.nslot * kPartStride * W;
                double accd[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) accd[q] = (double)accs[q] - (double)accc[q];
                item_partials<W, 3>(accd, sm, gslots + (size_t)blockIdx.x * kPartStride * W);
                if (tree_arrive<W, 3>(gslots, gridDim.x, blockIdx.x, a.bk_count + (size_t)gi * a.nbk,
                                      a.grp_count + gi, sm, red, &flag))
                    finish_group_a<W>(a.cs + P.col_off + (size_t)cur * W, first, red);
            }
            if (!have) break;
            cur = g;
            skip = a.grp_done[P.grp_off + g] != 0;
#pragma unroll
            for (int q = 0; q < 3; ++q) accs[q] = accc[q] = T(0);
            const ColState* csg = a.cs + P.col_off + (size_t)g * W;
            const int active = csg[cl].active;
            const double2 zd = csg[cl].z, bd = csg[cl].beta;
            z = cmk<V>((T)zd.x, (T)zd.y);
            beta = cmk<V>((T)bd.x, (T)bd.y);
            use_p = !first && active;
            const size_t tile = (size_t)P.vec_off + (size_t)g * n * W;
            rtile = (const char*)((const V*)a.r + tile);
            pl_ = (V*)a.p0 + tile + cl;
            ql_ = (V*)a.p1 + tile + cl;
        }
        if (skip) continue;
        const int rb = item - g * nrb;
        const int row0 = rb * RBW, row1 = min(n, row0 + RBW);
        if (tid < 32) {  // one lane per window issues its bulk copy; lanes 31, 30: entries, row pointers
            if (mrb != rb) {  // the table rows were not prefetched (first item, or skipped groups)
                mh = __ldg(a.whdr + rb);
                mwv = __ldg(a.wwin + (size_t)rb * kWinMax + (lane & (kWinMax - 1)));
                me0 = __ldg(app + row0);
            }
            const int4 h = mh;
            const int2 wv = lane < h.x ? mwv : make_int2(0, 0);
            int pos = wv.y;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, pos, o);
                if (lane >= o) pos += t;
            }
            pos -= wv.y;
            fence_proxy_async_smem();
            if (lane == 0) mbar_expect_tx(mb, (unsigned)h.y * ROWB + (unsigned)h.w * ENTB + LPP * 4u);
            __syncwarp();
            if (lane < h.x)
                bulk_g2s(xs_sh + (unsigned)pos * ROWB, rtile + (size_t)wv.x * ROWB, (unsigned)wv.y * ROWB, mb);
            if (lane == 31)
                bulk_g2s(lpp_sh, (const char*)a.wpk + (size_t)rb * LPP * 4 + (size_t)me0 * ENTB,
                         LPP * 4u + (unsigned)h.w * ENTB, mb);
            // the next item's table rows load while this item computes
            const int nx = item + gridDim.x;
            mrb = -1;
            if (nx < nitems) {
                mrb = nx % nrb;
                mh = __ldg(a.whdr + mrb);
                mwv = __ldg(a.wwin + (size_t)mrb * kWinMax + (lane & (kWinMax - 1)));
                me0 = __ldg(app + mrb * RBW);
            }
        }
        // own-row streams while the windows are in flight
        V po[RPT], qo[RPT];
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int i = row0 + rowslot + u * RPP;
            po[u] = zero;
            qo[u] = zero;
            if (use_p && i < row1) {
                po[u] = pl_[(size_t)i * W];
                qo[u] = ql_[(size_t)i * W];
            }
        }
        const bool ok = mbar_wait(mb, parity, a.wlimit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(a.werr, 1);
            mbar_wait(mb, parity, settle_limit(a.wlimit));  // let copies still in flight land before the CTA exits
            return;
        }
        parity ^= 1u;
        const int own0 = lp[RBW + 1];  // staged position of row0
        T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int i = row0 + rowslot + u * RPP;
            if (i < row1) {
                const int c0 = lp[i - row0], c1 = lp[i - row0 + 1];
                V ar = zero;
                for (int c = c0; c < c1; c += kChunk) {
                    int j[kChunk];
                    T av[kChunk];
                    load_chunk<T, true>(sent, c, j, av);
                    V xv[kChunk];
#pragma unroll
                    for (int v = 0; v < kChunk; ++v) xv[v] = j[v] >= 0 ? xs[(size_t)j[v] * W + cl] : zero;
#pragma unroll
                    for (int v = 0; v < kChunk; ++v) {
                        ar.x = fma(av[v], xv[v].x, ar.x);
                        ar.y = fma(av[v], xv[v].y, ar.y);
                    }
                }
                const V ri = xs[(size_t)(own0 + i - row0) * W + cl];
                V bx = ri;
                if (BM == 1) {
                    const T b = ((const T*)P.bd)[i];
                    bx = cmk<V>(b * ri.x, b * ri.y);
                }
                V pi_ = ri, qi = csub(cmul(z, bx), ar);  // (zB - A) r
                if (use_p) {
                    pi_ = cfma(beta, po[u], pi_);
                    qi = cfma(beta, qo[u], qi);
                }
                pl_[(size_t)i * W] = pi_;
                ql_[(size_t)i * W] = qi;
                acc[0] = fma(pi_.x, qi.x, fma(-pi_.y, qi.y, acc[0]));
                acc[1] = fma(pi_.x, qi.y, fma(pi_.y, qi.x, acc[1]));
                if (first) acc[2] = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[2]));
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) kahan_add(accs[q], accc[q], acc[q]);
        __syncthreads();  // staged rows and entries are free for the next item's copies
    }
}

// ---------------------------------------------------------------- warp-specialized staged step A
// The staged gathering step with the copies taken off the compute warps: one
// CTA per SM of 16 consumer warps and one producer warp, two stages.  The
// producer stages each item's windows of r, its own rows of p and q, its
// entries and its local row pointers (bulk copies onto the stage's "full"
// mbarrier) as soon as the consumers have released the stage (its "empty"
// mbarrier, one arrival per consumer warp), so the copies of the next item
// are in flight while the current one computes; the consumers only wait,
// compute and store.  Same arithmetic and partial sums as cocg_step_aw.
static constexpr int kThreadsWS = 512;          // consumer threads
static constexpr int kMaxGroupsWS = 1024;        // column groups per problem this kernel takes

__device__ __forceinline__ void mbar_arrive(unsigned addr)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}
// OR of pred over the kThreadsWS consumer threads (named barrier 1).
__device__ __forceinline__ bool consumers_or(bool pred)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((int)pred), "n"(kThreadsWS)
        : "memory");
    return r != 0;
}

template <typename T, int W, int BM, int RBW>
__global__ void __launch_bounds__(kThreadsWS + 32, 1) cocg_step_ws(FilterArgs a, int kk)
{
    const int k = a.kdev ? *a.kdev : kk;
    using V = c2_t<T>;
    using SY = NamedSync<1, kThreadsWS>;
    constexpr int NT = kThreadsWS;
    constexpr int RPP = NT / W;    // rows per pass of the consumers
    constexpr int RPT = RBW / RPP;  // rows per consumer thread per item
    static_assert(RBW % RPP == 0, "row block must be a whole number of passes");
    constexpr int LPP = RBW + 4;
    constexpr unsigned ROWB = W * sizeof(V);
    constexpr unsigned ENTB = sizeof(T) == 4 ? 8u : 16u;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ double sm[NT * 3];
    __shared__ double red[W * kPartStride];
    __shared__ int flag;
    __shared__ unsigned char s_done[kMaxGroupsWS];
    __shared__ __align__(8) unsigned long long mbar[4];  // full[0], full[1], empty[0], empty[1]
    const int tid = threadIdx.x, lane = tid & 31;
    const bool first = (k == 0);
    const FiltProb& P = a.probs[0];
    const int n = P.n, nrb = P.nrb, nitems = (int)a.nitems, G = P.G;
    const int* __restrict__ app = P.app;
    const unsigned cap = (unsigned)a.wcapr, cape = (unsigned)a.wcape;
    // a stage: [windows of r | own rows of p | own rows of q | entries | local row pointers]
    const unsigned p_off = cap * ROWB, q_off = p_off + RBW * ROWB, lpp_off = q_off + RBW * ROWB;
    const unsigned ent_off = lpp_off + LPP * 4u;  // staged metadata: row pointers, then entries
    const unsigned stage_bytes = (ent_off + cape * ENTB + 127u) & ~127u;
    const unsigned dsm_sh = (unsigned)__cvta_generic_to_shared(dsm);
    const unsigned base_sh = (dsm_sh + 127u) & ~127u;
    const unsigned char* base = dsm + (base_sh - dsm_sh);
    const unsigned mb0 = (unsigned)__cvta_generic_to_shared(&mbar[0]);  // full[s] = mb0 + 8s, empty[s] = mb0 + 16 + 8s
    if (tid == 0) {
        mbar_init(mb0, 1);
        mbar_init(mb0 + 8, 1);
        mbar_init(mb0 + 16, NT / 32);
        mbar_init(mb0 + 24, NT / 32);
        mbar_fence_init();
    }
    for (int g = tid; g < G; g += blockDim.x) s_done[g] = a.grp_done[P.grp_off + g] ? 1 : 0;
    __syncthreads();  // the last CTA-wide barrier: producer and consumers part here
    auto live_item = [&](int it) {
        while (it < nitems && s_done[it / nrb]) it += gridDim.x;
        return it;
    };

    if (tid >= NT) {  // ---- producer warp
        // table rows of the next item, loaded one item ahead
        int4 mh = make_int4(0, 0, 0, 0);
        int2 mwv = make_int2(0, 0);
        int me0 = 0;
        auto load_meta = [&](int it) {
            const int rb = it % nrb;
            mh = __ldg(a.whdr + rb);
            mwv = __ldg(a.wwin + (size_t)rb * kWinMax + (lane & (kWinMax - 1)));
            me0 = __ldg(app + rb * RBW);
        };
        int kq = 0;
        int it = live_item(blockIdx.x);
        if (it < nitems) load_meta(it);
        for (; it < nitems; ++kq) {
            const int st = kq & 1;
            const int4 h = mh;
            const int2 wv = lane < h.x ? mwv : make_int2(0, 0);
            const int e0 = me0;
            const int nx = live_item(it + gridDim.x);
            if (nx < nitems) load_meta(nx);
            if (kq >= 2) {  // the consumers released this stage (item kq - 2)
                if (!mbar_wait(mb0 + 16 + 8 * st, ((kq >> 1) - 1) & 1, a.wlimit)) {
                    if (lane == 0) atomicExch(a.werr, 1);
                    return;
                }
            }
            const int g = it / nrb, rb = it - g * nrb;
            const int row0 = rb * RBW, rows = min(n, row0 + RBW) - row0;
            int pos = wv.y;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, pos, o);
                if (lane >= o) pos += t;
            }
            pos -= wv.y;
            const size_t tile_b = ((size_t)P.vec_off + (size_t)g * n * W) * sizeof(V);
            const unsigned sb = base_sh + (unsigned)st * stage_bytes, full = mb0 + 8 * st;
            fence_proxy_async_smem();
            if (lane == 0)
                mbar_expect_tx(full, (unsigned)h.y * ROWB + (first ? 0u : 2u * rows * ROWB) + (unsigned)h.w * ENTB +
                                         LPP * 4u);
            __syncwarp();
            if (lane < h.x)
                bulk_g2s(sb + (unsigned)pos * ROWB, (const char*)a.r + tile_b + (size_t)wv.x * ROWB,
                         (unsigned)wv.y * ROWB, full);
            if (!first && lane == 16)
                bulk_g2s(sb + p_off, (const char*)a.p0 + tile_b + (size_t)row0 * ROWB, (unsigned)rows * ROWB, full);
            if (!first && lane == 17)
                bulk_g2s(sb + q_off, (const char*)a.p1 + tile_b + (size_t)row0 * ROWB, (unsigned)rows * ROWB, full);
            if (lane == 31)
                bulk_g2s(sb + lpp_off, (const char*)a.wpk + (size_t)rb * LPP * 4 + (size_t)e0 * ENTB,
                         LPP * 4u + (unsigned)h.w * ENTB, full);
            it = nx;
        }
        return;
    }

    // ---- consumer warps
    const int cl = tid % W, rowslot = tid / W;
    const V zero = cmk<V>(T(0), T(0));
    int cur = -1;
    bool use_p = false;
    V z = zero, beta = zero;
    V *pl_ = nullptr, *ql_ = nullptr;
    T accs[3] = {T(0), T(0), T(0)}, accc[3] = {T(0), T(0), T(0)};
    auto publish = [&](int g) {
        const int gi = P.grp_off + g;
        double* gslots = a.part + (size_t)gi * a.nslot * kPartStride * W;
        double accd[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) accd[q] = (double)accs[q] - (double)accc[q];
        item_partials<W, 3, double, NT, SY>(accd, sm, gslots + (size_t)blockIdx.x * kPartStride * W);
        if (tree_arrive<W, 3, NT, SY>(gslots, gridDim.x, blockIdx.x, a.bk_count + (size_t)gi * a.nbk,
                                      a.grp_count + gi, sm, red, &flag))
            finish_group_a<W>(a.cs + P.col_off + (size_t)g * W, first, red);
    };
    int kq = 0;
    for (int it = live_item(blockIdx.x); it < nitems; it = live_item(it + gridDim.x), ++kq) {
        const int g = it / nrb, rb = it - g * nrb;
        if (g != cur) {
            if (cur >= 0) publish(cur);
            cur = g;
#pragma unroll
            for (int q = 0; q < 3; ++q) accs[q] = accc[q] = T(0);
            const ColState* csg = a.cs + P.col_off + (size_t)g * W;
            const int active = csg[cl].active;
            const double2 zd = csg[cl].z, bd = csg[cl].beta;
            z = cmk<V>((T)zd.x, (T)zd.y);
            beta = cmk<V>((T)bd.x, (T)bd.y);
            use_p = !first && active;
            const size_t tile = (size_t)P.vec_off + (size_t)g * n * W;
            pl_ = (V*)a.p0 + tile + cl;
            ql_ = (V*)a.p1 + tile + cl;
        }
        const int st = kq & 1;
        const bool ok = mbar_wait(mb0 + 8 * st, (kq >> 1) & 1, a.wlimit);
        if (consumers_or(!ok)) {  // flag, then leave (all consumers) once the copies in flight have landed
            if (tid == 0) atomicExch(a.werr, 1);
            mbar_wait(mb0 + 8 * st, (kq >> 1) & 1, settle_limit(a.wlimit));
            mbar_wait(mb0 + 8 * (st ^ 1), ((kq + 1) >> 1) & 1, settle_limit(a.wlimit));
            return;
        }
        const unsigned char* sb = base + (unsigned)st * stage_bytes;
        const V* xs = (const V*)sb;
        const V* ps = (const V*)(sb + p_off);
        const V* qs = (const V*)(sb + q_off);
        const int4* sent = (const int4*)(sb + ent_off);
        const int* lp = (const int*)(sb + lpp_off);
        const int row0 = rb * RBW, row1 = min(n, row0 + RBW);
        const int own0 = lp[RBW + 1];
        T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int i = row0 + rowslot + u * RPP;
            if (i < row1) {
                const int c0 = lp[i - row0], c1 = lp[i - row0 + 1];
                V ar = zero;
                for (int c = c0; c < c1; c += kChunk) {
                    int j[kChunk];
                    T av[kChunk];
                    load_chunk<T, true>(sent, c, j, av);
                    V xv[kChunk];
#pragma unroll
                    for (int v = 0; v < kChunk; ++v) xv[v] = j[v] >= 0 ? xs[(size_t)j[v] * W + cl] : zero;
#pragma unroll
                    for (int v = 0; v < kChunk; ++v) {
                        ar.x = fma(av[v], xv[v].x, ar.x);
                        ar.y = fma(av[v], xv[v].y, ar.y);
                    }
                }
                const V ri = xs[(size_t)(own0 + i - row0) * W + cl];
                V bx = ri;
                if (BM == 1) {
                    const T b = ((const T*)P.bd)[i];
                    bx = cmk<V>(b * ri.x, b * ri.y);
                }
                V pi_ = ri, qi = csub(cmul(z, bx), ar);  // (zB - A) r
                if (use_p) {
                    pi_ = cfma(beta, ps[(size_t)(i - row0) * W + cl], pi_);
                    qi = cfma(beta, qs[(size_t)(i - row0) * W + cl], qi);
                }
                pl_[(size_t)i * W] = pi_;
                ql_[(size_t)i * W] = qi;
                acc[0] = fma(pi_.x, qi.x, fma(-pi_.y, qi.y, acc[0]));
                acc[1] = fma(pi_.x, qi.y, fma(pi_.y, qi.x, acc[1]));
                if (first) acc[2] = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[2]));
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) kahan_add(accs[q], accc[q], acc[q]);
        __syncwarp();
        if (lane == 0) mbar_arrive(mb0 + 16 + 8 * st);  // this warp is done with the stage
    }
    if (cur >= 0) publish(cur);
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
        const ItemInfo it = item_info(a, item);
        const FiltProb& P = a.probs[it.pi];
        const int g = it.g, rb = it.rb;
        if (!P.active) continue;
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
                ((T*)a.dQ)[P.dq_off + ((size_t)g * P.n + i) * a.mt + mloc] = T(0);
            }
        }
    }
}

// ---------------------------------------------------------------- standalone shifted SpMM
// V = (z B - A) P on the tiled layout: reads a.p0, writes a.p1.  Shifts come
// from the column states.
template <typename T, int W, int BM>
__global__ void __launch_bounds__(kThreads) shifted_spmm(FilterArgs a)
{
    using V = c2_t<T>;
    constexpr int RPP = kThreads / W;
    const int tid = threadIdx.x;
    const int cl = tid % W, rowslot = tid / W;
    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const ItemInfo it = item_info(a, item);
        const FiltProb& P = a.probs[it.pi];
        const double2 zd = a.cs[P.col_off + (size_t)it.g * W + cl].z;
        const V z = cmk<V>((T)zd.x, (T)zd.y);
        const size_t tile = (size_t)P.vec_off + (size_t)it.g * P.n * W;
        const V* x = (const V*)a.p0 + tile + cl;
        V* y = (V*)a.p1 + tile + cl;
        const int row0 = it.rb * a.RB;
        const int row1 = min(P.n, row0 + a.RB);
        for (int i = row0 + rowslot; i < row1; i += RPP) {
            V bx = __ldg(x + (size_t)i * W);
            const V ax = row_gather_global<T, W>(P.app, P.apk, i, x);
            if (BM == 1) {
                const T b = ((const T*)P.bd)[i];
                bx = cmk<V>(b * bx.x, b * bx.y);
            } else if (BM == 2) {
                bx = row_gather_global<T, W>(P.bpp, P.bpk, i, x);
            }
            y[(size_t)i * W] = csub(cmul(z, bx), ax);
        }
    }
}

// Step counter of graph-replayed COCG chunks: one thread adds one.
__global__ void k_advance(int* kdev) { *kdev += 1; }

cudaError_t launch_advance(int* kdev, cudaStream_t s)
{
    k_advance<<<1, 1, 0, s>>>(kdev);
    count_launches(1);
    return cudaGetLastError();
}

// Q += dQ after all node batches of a pass (dQ: FP32 in mixed precision,
// tiled [group][row][mt] per problem; Q row-major n x m0 per problem).
template <typename T>
__global__ void fold_dq(const FiltProb* probs, int nprob, int mt, const T* dQ, double* Q)
{
    const FiltProb& P = probs[blockIdx.y];
    if (!P.active) return;
    const long long total = (long long)P.n * P.m0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / P.m0), m = (int)(t % P.m0);
        const int g = m / mt, ml = m % mt;
        Q[P.q_off + t] += (double)dQ[P.dq_off + ((size_t)g * P.n + i) * mt + ml];
    }
}

// Packed (column, value) CSR entries padded to whole chunks: row i occupies
// entries [pp[i], pp[i+1]) of out, its (first) diagonal entry first, then the
// other stored entries in order; entries past the row's nonzeros are (-1, 0).
// One warp per row.
__global__ void pack_csr(int n, const int* ia, const int* ja, const double* av, const int* pp, int fp64, void* out)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nw) {
        const int s = ia[i], len = ia[i + 1] - s, c0 = pp[i], c1 = pp[i + 1];
        // position of the row's (first) diagonal entry, -1 if it has none
        int dpos = -1;
        for (int base = 0; base < len; base += 32) {
            const int t = base + lane;
            const unsigned b = __ballot_sync(0xffffffffu, t < len && ja[s + t] == i);
            if (b) {
                dpos = base + __ffs(b) - 1;
                break;
            }
        }
        for (int t = c0 + lane; t < c1; t += 32) {
            const int q = t - c0;
            // diagonal first, then the other entries in their stored order
            int src = -1;
            if (q < len) src = dpos < 0 ? q : (q == 0 ? dpos : (q - 1 < dpos ? q - 1 : q));
            const int j = src >= 0 ? ja[s + src] : -1;
            const double v = src >= 0 ? av[s + src] : 0.0;
            if (fp64) ((int4*)out)[t] = make_int4(j, 0, __double2loint(v), __double2hiint(v));
            else ((int2*)out)[t] = make_int2(j, __float_as_int((float)v));
        }
    }
}

__global__ void cast_diag(int n, const int* ia, const double* av, int fp64, void* out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = av[ia[i]];
        if (fp64) ((double*)out)[i] = v;
        else ((float*)out)[i] = (float)v;
    }
}

cudaError_t launch_fold_dq(const FilterArgs& a, long long max_total, bool fp64, cudaStream_t s)
{
    if (max_total <= 0) return cudaSuccess;
    long long blocks = (max_total + 255) / 256;
    if (blocks > (long long)num_sms() * 8) blocks = (long long)num_sms() * 8;
    dim3 grid((unsigned)blocks, a.nprob);
    if (fp64) fold_dq<double><<<grid, 256, 0, s>>>(a.probs, a.nprob, a.mt, (const double*)a.dQ, a.Q);
    else fold_dq<float><<<grid, 256, 0, s>>>(a.probs, a.nprob, a.mt, (const float*)a.dQ, a.Q);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack_csr(int n, const int* ia, const int* ja, const double* av, const int* pp, bool fp64, void* out,
                            cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = ((long long)n + 7) / 8;
    if (blocks > 4096) blocks = 4096;
    pack_csr<<<(int)blocks, 256, 0, s>>>(n, ia, ja, av, pp, fp64 ? 1 : 0, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cast_diag(int n, const int* ia, const double* av, bool fp64, void* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = ((long long)n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    cast_diag<<<(int)blocks, 256, 0, s>>>(n, ia, av, fp64 ? 1 : 0, out);
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

#define FEAST_LAUNCH_T(KERNEL, T, BMV, ...)                                          \
    do {                                                                             \
        if (a.W == 16) KERNEL<T, 16, BMV><<<grid, kThreads, 0, s>>>(__VA_ARGS__);    \
        else if (a.W == 32) KERNEL<T, 32, BMV><<<grid, kThreads, 0, s>>>(__VA_ARGS__); \
        else return cudaErrorInvalidValue;                                           \
    } while (0)

#define FEAST_DISPATCH_B(KERNEL, ...)                                                \
    do {                                                                             \
        if (fp64) {                                                                  \
            if (a.bmode == 0) FEAST_LAUNCH_T(KERNEL, double, 0, __VA_ARGS__);        \
            else if (a.bmode == 1) FEAST_LAUNCH_T(KERNEL, double, 1, __VA_ARGS__);   \
            else FEAST_LAUNCH_T(KERNEL, double, 2, __VA_ARGS__);                     \
        } else {                                                                     \
            if (a.bmode == 0) FEAST_LAUNCH_T(KERNEL, float, 0, __VA_ARGS__);         \
            else if (a.bmode == 1) FEAST_LAUNCH_T(KERNEL, float, 1, __VA_ARGS__);    \
            else FEAST_LAUNCH_T(KERNEL, float, 2, __VA_ARGS__);                      \
        }                                                                            \
        count_launches(1);                                                           \
        return cudaGetLastError();                                                   \
    } while (0)

cudaError_t launch_cocg_step_a(const FilterArgs& a, bool fp64, int k, int grid, cudaStream_t s)
{
    FEAST_DISPATCH_B(cocg_step_a, a, k);
}

cudaError_t launch_cocg_step_b(const FilterArgs& a, bool fp64, int k, int grid, cudaStream_t s)
{
    FEAST_DISPATCH_B(cocg_step_b, a, k);
}

// ---------------------------------------------------------------- staged-window launchers
cudaError_t launch_win_build(int n, int rbw, const int* pp, const void* pk, bool fp64, void* meta, int4* hdr,
                             int2* win, int* stat, cudaStream_t s)
{
    if (n <= 0 || rbw <= 0) return cudaSuccess;
    const int nrbw = (n + rbw - 1) / rbw;
    const int grid = std::min(nrbw, num_sms() * 8);
    if (fp64)
        win_build<int4><<<grid, 256, 0, s>>>(n, rbw, nrbw, pp, (const int4*)pk, (char*)meta, hdr, win, stat);
    else
        win_build<int2><<<grid, 256, 0, s>>>(n, rbw, nrbw, pp, (const int2*)pk, (char*)meta, hdr, win, stat);
    count_launches(1);
    return cudaGetLastError();
}

size_t win_smem_bytes(bool fp64, int W, int rbw, int capr, int cape)
{
    const size_t cb = fp64 ? 16 : 8;  // complex element, and packed entry, bytes
    // + alignment pad of the staged rows; the local row pointers last
    return 128 + (size_t)capr * W * cb + (size_t)cape * cb + (size_t)(rbw + 4) * 4;
}

// Allows the variant the largest dynamic shared memory the device gives a CTA
// (idempotent), then returns its resident CTAs per SM at `smem` bytes.
template <typename T, int W, int BM, int RBW>
static int aw_occupancy(size_t smem)
{
    auto kern = cocg_step_aw<T, W, BM, RBW>;
    cudaFuncAttributes fa;
    int dev = 0, optin = 0;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const long long room = (long long)optin - (long long)fa.sharedSizeBytes;
    if (room <= 0 || (long long)smem > room) return 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return o;
}

template <typename T, int W>
static int aw_occupancy_tw(int bmode, int rbw, size_t smem)
{
    if (sizeof(T) == 4 && bmode == 0 && rbw == 80) return aw_occupancy<T, W, 0, 80>(smem);
    if (sizeof(T) == 4 && bmode == 1 && rbw == 80) return aw_occupancy<T, W, 1, 80>(smem);
    if (bmode == 0 && rbw == 64) return aw_occupancy<T, W, 0, 64>(smem);
    if (bmode == 0 && rbw == 32) return aw_occupancy<T, W, 0, 32>(smem);
    if (bmode == 1 && rbw == 64) return aw_occupancy<T, W, 1, 64>(smem);
    if (bmode == 1 && rbw == 32) return aw_occupancy<T, W, 1, 32>(smem);
    return 0;
}

// Variants built: complex FP32 with 32 lanes, complex FP64 with 16 lanes (a
// 256-byte tile row each); B the identity or diagonal; 32 or 64 rows per item,
// and 80 for complex FP32.
int win_occupancy(bool fp64, int W, int bmode, int rbw, size_t smem)
{
    if (!fp64 && W == 32) return aw_occupancy_tw<float, 32>(bmode, rbw, smem);
    if (fp64 && W == 16) return aw_occupancy_tw<double, 16>(bmode, rbw, smem);
    return 0;
}

template <typename T, int W>
static cudaError_t aw_launch_tw(const FilterArgs& a, int rbw, int k, int grid, size_t smem, cudaStream_t s)
{
    if (sizeof(T) == 4 && a.bmode == 0 && rbw == 80) cocg_step_aw<T, W, 0, 80><<<grid, kThreads, smem, s>>>(a, k);
    else if (sizeof(T) == 4 && a.bmode == 1 && rbw == 80) cocg_step_aw<T, W, 1, 80><<<grid, kThreads, smem, s>>>(a, k);
    else if (a.bmode == 0 && rbw == 64) cocg_step_aw<T, W, 0, 64><<<grid, kThreads, smem, s>>>(a, k);
    else if (a.bmode == 0 && rbw == 32) cocg_step_aw<T, W, 0, 32><<<grid, kThreads, smem, s>>>(a, k);
    else if (a.bmode == 1 && rbw == 64) cocg_step_aw<T, W, 1, 64><<<grid, kThreads, smem, s>>>(a, k);
    else if (a.bmode == 1 && rbw == 32) cocg_step_aw<T, W, 1, 32><<<grid, kThreads, smem, s>>>(a, k);
    else return cudaErrorInvalidValue;
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cocg_step_aw(const FilterArgs& a, bool fp64, int rbw, int k, int grid, size_t smem,
                                cudaStream_t s)
{
    if (!fp64 && a.W == 32) return aw_launch_tw<float, 32>(a, rbw, k, grid, smem, s);
    if (fp64 && a.W == 16) return aw_launch_tw<double, 16>(a, rbw, k, grid, smem, s);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- warp-specialized step A launchers
size_t ws_smem_bytes(int W, int rbw, int capr, int cape)
{
    const size_t rowb = (size_t)W * 8;  // complex FP32 tiles
    const size_t stage = ((size_t)capr * rowb + 2 * (size_t)rbw * rowb + (size_t)cape * 8 + (size_t)(rbw + 4) * 4 + 127) &
                         ~(size_t)127;
    return 128 + 2 * stage;
}

template <int BM, int RBW>
static int ws_occupancy_one(size_t smem)
{
    auto kern = cocg_step_ws<float, 32, BM, RBW>;
    cudaFuncAttributes fa;
    int dev = 0, optin = 0;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const long long room = (long long)optin - (long long)fa.sharedSizeBytes;
    if (room <= 0 || (long long)smem > room) return 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kThreadsWS + 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return o;
}

// Variants built: complex FP32, 32 lanes, B the identity or diagonal, 48 or 32
// rows per item; at most kMaxGroupsWS column groups.
int ws_occupancy(bool fp64, int W, int bmode, int rbw, int groups, size_t smem)
{
    if (fp64 || W != 32 || groups > kMaxGroupsWS) return 0;
    if (bmode == 0 && rbw == 48) return ws_occupancy_one<0, 48>(smem);
    if (bmode == 0 && rbw == 32) return ws_occupancy_one<0, 32>(smem);
    if (bmode == 1 && rbw == 48) return ws_occupancy_one<1, 48>(smem);
    if (bmode == 1 && rbw == 32) return ws_occupancy_one<1, 32>(smem);
    return 0;
}

cudaError_t launch_cocg_step_ws(const FilterArgs& a, int rbw, int k, int grid, size_t smem, cudaStream_t s)
{
    if (a.W != 32) return cudaErrorInvalidValue;
    if (a.bmode == 0 && rbw == 48) cocg_step_ws<float, 32, 0, 48><<<grid, kThreadsWS + 32, smem, s>>>(a, k);
    else if (a.bmode == 0 && rbw == 32) cocg_step_ws<float, 32, 0, 32><<<grid, kThreadsWS + 32, smem, s>>>(a, k);
    else if (a.bmode == 1 && rbw == 48) cocg_step_ws<float, 32, 1, 48><<<grid, kThreadsWS + 32, smem, s>>>(a, k);
    else if (a.bmode == 1 && rbw == 32) cocg_step_ws<float, 32, 1, 32><<<grid, kThreadsWS + 32, smem, s>>>(a, k);
    else return cudaErrorInvalidValue;
    count_launches(1);
    return cudaGetLastError();
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
    FEAST_DISPATCH_B(shifted_spmm, a);
}

// Persistent grid sizes of the COCG launches: SMs x resident CTAs per SM of
// each kernel (identity-B variants; the others differ little).
void filter_grids(bool fp64, int W, int* grid_a, int* grid_b)
{
    int oa = 0, ob = 0;
    if (fp64) {
        if (W == 16) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oa, cocg_step_a<double, 16, 0>, kThreads, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, cocg_step_b<double, 16, 0>, kThreads, 0);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oa, cocg_step_a<double, 32, 0>, kThreads, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, cocg_step_b<double, 32, 0>, kThreads, 0);
        }
    } else {
        if (W == 16) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oa, cocg_step_a<float, 16, 0>, kThreads, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, cocg_step_b<float, 16, 0>, kThreads, 0);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oa, cocg_step_a<float, 32, 0>, kThreads, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, cocg_step_b<float, 32, 0>, kThreads, 0);
        }
    }
    cudaGetLastError();
    if (oa < 1) oa = 1;
    if (ob < 1) ob = 1;
    *grid_a = num_sms() * oa;
    *grid_b = num_sms() * ob;
}

int filter_grid(bool fp64, int W)
{
    int ga, gb;
    filter_grids(fp64, W, &ga, &gb);
    return ga > gb ? ga : gb;
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
