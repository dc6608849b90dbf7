// Batched Rayleigh-Ritz for many independent eigenproblems of uneven size
// (FEAST v4.0 guide, Sec. 1.1: one reduced problem per search interval; the
// guide's parallelism level L1 runs separate intervals independently).
//
// Every kernel here covers all problems of a batch in one launch: rows of all
// problems are flattened into one index space (or work blocks are listed per
// problem), and a problem table (BProb) gives each problem's sizes and
// offsets.  A problem whose flag `active` is 0 is skipped, so one launch
// sequence (and one captured CUDA graph) serves every refinement loop while
// problems converge at different loops.
//
//   b_spmm        Y = A X for every problem's FP64 row-major n x m block
//   b_gram        partial C = X^T Y per (problem, 64x64 tile pair, row split),
//                 FP64 tensor cores (mma.sync m8n8k4 f64); b_gram_reduce sums
//                 the splits in order and symmetrises
//   b_gemm        C = A V (n x m times m x m) per problem
//   b_residual    R = A X - B X diag(lambda) and per-column norms
//   b_reduced     the reduced generalized eigenproblem of one problem per CTA
//                 (m <= 128): two cyclic Jacobi decompositions in shared and
//                 global memory, rounds synchronised with __syncthreads
#include "chol.cuh"
#include "feast_internal.cuh"

namespace feast {

static constexpr int BT = 64, BK = 16, BLD = BT + 4;
static constexpr int kRedThreads = 512;
static constexpr double kSentinelB = 1e300;

template <typename F>
__device__ __forceinline__ int bsearch_ll(const BProb* pr, int np, long long key, F field)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (field(pr[mid]) <= key) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- SpMM
__global__ void __launch_bounds__(256) b_spmm(const BProb* pr, int np, long long rows, const double* __restrict__ X,
                                             double* __restrict__ Y, int useB)
{
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long gr = warp; gr < rows; gr += nw) {
        const int p = bsearch_ll(pr, np, gr, [](const BProb& b) { return b.row0; });
        const BProb& P = pr[p];
        if (!P.active) continue;
        const int i = (int)(gr - P.row0), m = P.m;
        const int* ia = useB ? P.ib : P.ia;
        const int* ja = useB ? P.jb : P.ja;
        const double* av = useB ? P.bv : P.av;
        const double* Xp = X + P.q_off;
        double* Yp = Y + P.q_off;
        const int s = ia[i], e = ia[i + 1];
        for (int c0 = 0; c0 < m; c0 += 32) {
            const int c = c0 + lane;
            double acc = 0.0;
            for (int t = s; t < e; ++t) {
                const int j = __ldg(ja + t);
                const double a = __ldg(av + t);
                if (c < m) acc = fma(a, __ldg(Xp + (size_t)j * m + c), acc);
            }
            if (c < m) Yp[(size_t)i * m + c] = acc;
        }
    }
}

// ---------------------------------------------------------------- FP64 tensor-core tiles
__device__ __forceinline__ void bdmma(double& c0, double& c1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

__device__ __forceinline__ void btile_mma(const double (*As)[BLD], const double (*Bs)[BLD], double (&acc)[4][4][2],
                                          int wr, int wc, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < BK; kk += 4) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk + t][wr + i * 8 + g];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk + t][wc + j * 8 + g];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) bdmma(acc[i][j][0], acc[i][j][1], a[i], b[j]);
    }
}

// block -> (problem, upper tile (ta <= tb), split); partial tile of X^T Y
__global__ void __launch_bounds__(128) b_gram(const BProb* pr, int np, int nblocks, const double* __restrict__ X,
                                              const double* __restrict__ Y, double* __restrict__ part)
{
    __shared__ __align__(16) double As[BK][BLD];
    __shared__ __align__(16) double Bs[BK][BLD];
    const int blk = blockIdx.x;
    if (blk >= nblocks) return;
    const int p = bsearch_ll(pr, np, blk, [](const BProb& b) { return (long long)b.gram_b0; });
    const BProb& P = pr[p];
    if (!P.active) return;
    const int local = blk - P.gram_b0;
    const int tile = local / P.gram_ks, split = local % P.gram_ks;
    int t = tile, ta = 0;
    while (t >= P.gram_T - ta) { t -= P.gram_T - ta; ++ta; }
    const int tb = ta + t;
    const int m = P.m, n = P.n;
    const int a0 = ta * BT, b0 = tb * BT;
    const long long chunk = ((long long)n + P.gram_ks - 1) / P.gram_ks;
    const int r0 = (int)min((long long)n, split * chunk), r1 = (int)min((long long)n, (split + 1) * chunk);
    const double* Xp = X + P.q_off;
    const double* Yp = Y + P.q_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    for (int k0 = r0; k0 < r1; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int idx = tid + q * 128;
            const int kk = idx >> 6, c = idx & 63;
            const int r = k0 + kk;
            const bool rok = r < r1;
            As[kk][c] = (rok && a0 + c < m) ? __ldg(Xp + (size_t)r * m + a0 + c) : 0.0;
            Bs[kk][c] = (rok && b0 + c < m) ? __ldg(Yp + (size_t)r * m + b0 + c) : 0.0;
        }
        __syncthreads();
        btile_mma(As, Bs, acc, wr, wc, lane);
        __syncthreads();
    }
    double* out = part + P.gpart_off + (size_t)split * m * m;
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int row = a0 + wr + i * 8 + g;
            const int col = b0 + wc + j * 8 + 2 * tq;
            if (row < m && col < m) out[(size_t)row * m + col] = acc[i][j][0];
            if (row < m && col + 1 < m) out[(size_t)row * m + col + 1] = acc[i][j][1];
        }
}

// C (m x m per problem at c_off) from the partial tiles; grid.y = problem
__global__ void b_gram_reduce(const BProb* pr, const double* __restrict__ part, double* __restrict__ C)
{
    const BProb& P = pr[blockIdx.y];
    if (!P.active) return;
    const int m = P.m, ks = P.gram_ks;
    const double* pp = part + P.gpart_off;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
        const int i = idx / m, j = idx % m;
        const int ti = i / BT, tj = j / BT;
        double v;
        if (ti == tj) {
            double s1 = 0.0, s2 = 0.0;
            for (int s = 0; s < ks; ++s) {
                s1 += pp[(size_t)s * m * m + (size_t)i * m + j];
                s2 += pp[(size_t)s * m * m + (size_t)j * m + i];
            }
            v = 0.5 * (s1 + s2);
        } else {
            const int a = ti < tj ? i : j, b = ti < tj ? j : i;
            double s1 = 0.0;
            for (int s = 0; s < ks; ++s) s1 += pp[(size_t)s * m * m + (size_t)a * m + b];
            v = s1;
        }
        C[P.c_off + idx] = v;
    }
}

// Out = A V per problem: A (n x m at q_off), V (m x m at c_off), Out (n x m at q_off)
__global__ void __launch_bounds__(128) b_gemm(const BProb* pr, int np, int nblocks, const double* __restrict__ A,
                                              const double* __restrict__ V, double* __restrict__ Out)
{
    __shared__ __align__(16) double As[BK][BLD];
    __shared__ __align__(16) double Bs[BK][BLD];
    const int blk = blockIdx.x;
    if (blk >= nblocks) return;
    const int p = bsearch_ll(pr, np, blk, [](const BProb& b) { return (long long)b.gemm_b0; });
    const BProb& P = pr[p];
    if (!P.active) return;
    const int m = P.m, n = P.n;
    const int ct = (m + BT - 1) / BT;
    const int local = blk - P.gemm_b0;
    const int r0 = (local / ct) * BT, c0 = (local % ct) * BT;
    const double* Ap = A + P.q_off;
    const double* Vp = V + P.c_off;
    double* Op = Out + P.q_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    for (int k0 = 0; k0 < m; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int idx = tid + q * 128;
            const int ar = idx >> 4, ak = idx & 15;
            const int gr = r0 + ar, gk = k0 + ak;
            As[ak][ar] = (gr < n && gk < m) ? __ldg(Ap + (size_t)gr * m + gk) : 0.0;
            const int bk = idx >> 6, bc = idx & 63;
            const int vk = k0 + bk, vc = c0 + bc;
            Bs[bk][bc] = (vk < m && vc < m) ? __ldg(Vp + (size_t)vk * m + vc) : 0.0;
        }
        __syncthreads();
        btile_mma(As, Bs, acc, wr, wc, lane);
        __syncthreads();
    }
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int row = r0 + wr + i * 8 + g;
            const int col = c0 + wc + j * 8 + 2 * tq;
            if (row < n && col < m) Op[(size_t)row * m + col] = acc[i][j][0];
            if (row < n && col + 1 < m) Op[(size_t)row * m + col + 1] = acc[i][j][1];
        }
}

// ---------------------------------------------------------------- residuals
// block -> (problem, 256-row block); per-column partial sums of R^2, (Bx)^2
static constexpr int kResRows = 256;

__global__ void __launch_bounds__(256) b_residual(const BProb* pr, int np, int nblocks, const double* __restrict__ X,
                                                  const double* __restrict__ lam, double* __restrict__ R,
                                                  double* __restrict__ part)
{
    __shared__ double sr[8][128];
    __shared__ double sb[8][128];
    const int blk = blockIdx.x;
    if (blk >= nblocks) return;
    const int p = bsearch_ll(pr, np, blk, [](const BProb& b) { return (long long)b.res_b0; });
    const BProb& P = pr[p];
    if (!P.active) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = P.m, n = P.n;
    const int rb = blk - P.res_b0;
    const double* Xp = X + P.q_off;
    double* Rp = R + P.q_off;
    const double* lp = lam + P.l_off;
    double accr[4] = {0, 0, 0, 0}, accb[4] = {0, 0, 0, 0};
    for (int i = rb * kResRows + warp; i < min(n, (rb + 1) * kResRows); i += 8) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = q * 32 + lane;
            if (c >= m) continue;
            double ax = 0.0, bx = 0.0;
            for (int t = P.ia[i]; t < P.ia[i + 1]; ++t) ax = fma(__ldg(P.av + t), __ldg(Xp + (size_t)__ldg(P.ja + t) * m + c), ax);
            if (P.ib) {
                for (int t = P.ib[i]; t < P.ib[i + 1]; ++t) bx = fma(__ldg(P.bv + t), __ldg(Xp + (size_t)__ldg(P.jb + t) * m + c), bx);
            } else {
                bx = Xp[(size_t)i * m + c];
            }
            const double r = fma(-lp[c], bx, ax);
            Rp[(size_t)i * m + c] = r;
            accr[q] = fma(r, r, accr[q]);
            accb[q] = fma(bx, bx, accb[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        sr[warp][q * 32 + lane] = accr[q];
        sb[warp][q * 32 + lane] = accb[q];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        double s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < 8; ++w) { s1 += sr[w][c]; s2 += sb[w][c]; }
        part[((size_t)blk * 128 + c) * 2] = s1;
        part[((size_t)blk * 128 + c) * 2 + 1] = s2;
    }
}

// grid.y = problem; res[c] = ||R_c|| / (alpha ||B x_c||)
__global__ void b_residual_cols(const BProb* pr, const double* __restrict__ part, double* __restrict__ res)
{
    const BProb& P = pr[blockIdx.y];
    if (!P.active) return;
    const int nrb = (P.n + kResRows - 1) / kResRows;
    for (int c = threadIdx.x; c < P.m; c += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int rb = 0; rb < nrb; ++rb) {
            a += part[((size_t)(P.res_b0 + rb) * 128 + c) * 2];
            b += part[((size_t)(P.res_b0 + rb) * 128 + c) * 2 + 1];
        }
        const double bn = sqrt(b);
        res[P.l_off + c] = bn > 0.0 ? sqrt(a) / (P.alpha * bn) : 0.0;
    }
}

// ---------------------------------------------------------------- reduced problem, one CTA per problem
struct CtaRot {
    double c[64], s[64], t[64];
    int p[64], q[64];
    double red[kRedThreads];
    int flag;
};

// Cyclic Jacobi (round-robin pairs) on the m x m row-major matrix A (m <= 128)
// in global memory, eigenvectors accumulated in V; rotations below the
// relative threshold are skipped; ends with diag(A) holding the eigenvalues.
__device__ void cta_jacobi(int m, double* A, double* V, CtaRot& R)
{
    const int mp = m + (m & 1), half = mp / 2;
    double part = 0.0;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
        V[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
        part += fabs(A[idx]) < 1e299 ? A[idx] * A[idx] : 0.0;  // sentinels excluded
    }
    R.red[threadIdx.x] = part;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) R.red[threadIdx.x] += R.red[threadIdx.x + o];
        __syncthreads();
    }
    const double absfloor = 1e-18 * sqrt(R.red[0]);
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (threadIdx.x == 0) R.flag = 0;
        __syncthreads();
        for (int r = 0; r < mp - 1; ++r) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int p = k == 0 ? 0 : 1 + (k - 1 + r) % (mp - 1);
                const int s2 = mp - 1 - k;
                int q = s2 == 0 ? 0 : 1 + (s2 - 1 + r) % (mp - 1);
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0, tt = 0.0;
                if (q < m) {
                    const double apq = A[p * m + q], app = A[p * m + p], aqq = A[q * m + q];
                    const double thr = fmax(1.1e-16 * sqrt(fabs(app * aqq)), absfloor);
                    if (fabs(apq) > thr) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                        R.flag = 1;
                    }
                }
                R.c[k] = c;
                R.s[k] = s;
                R.t[k] = tt;
                R.p[k] = p;
                R.q[k] = q;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < half * half; idx += blockDim.x) {
                const int k = idx / half, l = idx % half;
                const double ck = R.c[k], sk = R.s[k], cl = R.c[l], sl = R.s[l];
                if (sk == 0.0 && sl == 0.0) continue;
                const int p = R.p[k], q = R.q[k], pp = R.p[l], qq = R.q[l];
                if (k == l) {
                    const double apq = A[p * m + q], tt = R.t[k];
                    A[p * m + p] -= tt * apq;
                    A[q * m + q] += tt * apq;
                    A[p * m + q] = 0.0;
                    A[q * m + p] = 0.0;
                    continue;
                }
                const bool qv = q < m, qqv = qq < m;
                const double x00 = A[p * m + pp];
                const double x01 = qqv ? A[p * m + qq] : 0.0;
                const double x10 = qv ? A[q * m + pp] : 0.0;
                const double x11 = (qv && qqv) ? A[q * m + qq] : 0.0;
                const double y00 = ck * x00 - sk * x10, y01 = ck * x01 - sk * x11;
                const double y10 = sk * x00 + ck * x10, y11 = sk * x01 + ck * x11;
                A[p * m + pp] = cl * y00 - sl * y01;
                if (qqv) A[p * m + qq] = sl * y00 + cl * y01;
                if (qv) A[q * m + pp] = cl * y10 - sl * y11;
                if (qv && qqv) A[q * m + qq] = sl * y10 + cl * y11;
            }
            for (int idx = threadIdx.x; idx < m * half; idx += blockDim.x) {
                const int i = idx / half, k = idx % half;
                const double sk = R.s[k];
                if (sk == 0.0) continue;
                const double ck = R.c[k];
                const int p = R.p[k], q = R.q[k];
                const double vp = V[i * m + p], vq = V[i * m + q];
                V[i * m + p] = ck * vp - sk * vq;
                V[i * m + q] = sk * vp + ck * vq;
            }
            __syncthreads();
        }
        const int any = R.flag;
        __syncthreads();
        if (!any) break;
    }
}

// Reduced generalized problem of one problem per CTA (m <= 128): scale by
// D = diag(B_Q)^{-1/2}; S = D L^{-T} from B~ = L L^T when the Cholesky
// factor is accepted, else Jacobi on B~, keep d > 1e-14 max d,
// S = D U_k d_k^{-1/2} (sentinel on dropped directions); C = S^T A~ S,
// Jacobi on C, V = S W; lam
// ascending (live values first), mk live count.  work: 6 m*m + 4 m doubles.
__global__ void __launch_bounds__(kRedThreads) b_reduced(const BProb* pr, const double* __restrict__ Aq,
                                                          const double* __restrict__ Bq, double* __restrict__ lam,
                                                          double* __restrict__ Vout, int* __restrict__ mk,
                                                          double* __restrict__ work)
{
    __shared__ CtaRot R;
    const BProb& P = pr[blockIdx.x];
    if (!P.active) return;
    const int m = P.m;
    const size_t mm = (size_t)m * m;
    double* W0 = work + P.w_off;
    double* At = W0;
    double* Bt = At + mm;
    double* U = Bt + mm;
    double* S = U + mm;
    double* C = S + mm;
    double* Wv = C + mm;
    double* dsc = Wv + mm;
    double* d = dsc + m;
    const double* aq = Aq + P.c_off;
    const double* bq = Bq + P.c_off;
    for (int idx = threadIdx.x; idx < (int)mm; idx += blockDim.x) {
        const int i = idx / m, j = idx % m;
        const double bi = bq[i * m + i], bj = bq[j * m + j];
        const double di = bi > 0.0 ? 1.0 / sqrt(bi) : 0.0, dj = bj > 0.0 ? 1.0 / sqrt(bj) : 0.0;
        Bt[idx] = 0.5 * (bq[i * m + j] + bq[j * m + i]) * di * dj;
        At[idx] = 0.5 * (aq[i * m + j] + aq[j * m + i]);
        if (j == 0) dsc[i] = di;
    }
    for (int idx = threadIdx.x; idx < (int)mm; idx += blockDim.x) U[idx] = Bt[idx];
    __syncthreads();
    double* xd = d + m;
    const bool chol = cta_chol_inv(m, U, xd, d + 2 * m, R.red);
    int live = m;
    if (chol) {  // S = D L^{-T}
        for (int idx = threadIdx.x; idx < (int)mm; idx += blockDim.x) {
            const int r = idx / m, c = idx % m;
            S[idx] = c > r ? dsc[r] * U[idx] : (c == r ? dsc[r] * xd[r] : 0.0);
        }
    } else {
        cta_jacobi(m, Bt, U, R);
        __syncthreads();
        double dmax = 0.0;
        for (int i = 0; i < m; ++i) dmax = fmax(dmax, Bt[i * m + i]);
        for (int i = threadIdx.x; i < m; i += blockDim.x) d[i] = Bt[i * m + i];
        __syncthreads();
        for (int idx = threadIdx.x; idx < (int)mm; idx += blockDim.x) {
            const int r = idx / m, c = idx % m;
            const bool keep = dmax > 0.0 && d[c] > 1e-14 * dmax;
            S[idx] = keep ? dsc[r] * U[idx] / sqrt(d[c]) : 0.0;
        }
        live = 0;
        for (int c = 0; c < m; ++c) live += (dmax > 0.0 && d[c] > 1e-14 * dmax);
    }
    __syncthreads();
    // T = A~ S into U, then C = S^T T
    for (int idx = threadIdx.x; idx < (int)mm; idx += blockDim.x) {
        const int r = idx / m, c = idx % m;
        double s = 0.0;
        for (int l = 0; l < m; ++l) s = fma(At[r * m + l], S[l * m + c], s);
        U[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < (int)mm; idx += blockDim.x) {
        const int r = idx / m, c = idx % m;
        if (c < r) continue;
        double s = 0.0;
        for (int l = 0; l < m; ++l) s = fma(S[l * m + r], U[l * m + c], s);
        C[r * m + c] = s;
        C[c * m + r] = s;
    }
    __syncthreads();
    if (!chol) {
        for (int c = threadIdx.x; c < m; c += blockDim.x) {
            bool zero = true;
            for (int r = 0; r < m && zero; ++r) zero = S[r * m + c] == 0.0;
            if (zero) C[c * m + c] = kSentinelB;
        }
    }
    __syncthreads();
    cta_jacobi(m, C, Wv, R);
    __syncthreads();
    // V = S W with columns sorted by ascending eigenvalue
    double* lp = lam + P.l_off;
    double* vo = Vout + P.c_off;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double li = C[i * m + i];
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double lj = C[j * m + j];
            rank += (lj < li) || (lj == li && j < i);
        }
        lp[rank] = li;
        for (int r = 0; r < m; ++r) {
            double s = 0.0;
            for (int l = 0; l < m; ++l) s = fma(S[r * m + l], Wv[l * m + i], s);
            vo[r * m + rank] = s;
        }
    }
    if (threadIdx.x == 0) mk[blockIdx.x] = live;
}

// ---------------------------------------------------------------- launchers
static int cap_blocks(long long want, int per_sm)
{
    const long long cap = (long long)num_sms() * per_sm;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

cudaError_t launch_b_spmm(const BProb* pr, int np, long long rows, const double* X, double* Y, int useB, cudaStream_t s)
{
    b_spmm<<<cap_blocks((rows + 7) / 8, 16), 256, 0, s>>>(pr, np, rows, X, Y, useB);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_b_gram(const BProb* pr, int np, int nblocks, int maxm, const double* X, const double* Y, double* part,
                          double* C, cudaStream_t s)
{
    if (nblocks > 0) b_gram<<<nblocks, 128, 0, s>>>(pr, np, nblocks, X, Y, part);
    dim3 g((unsigned)((maxm * maxm + 255) / 256), np);
    b_gram_reduce<<<g, 256, 0, s>>>(pr, part, C);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_b_gemm(const BProb* pr, int np, int nblocks, const double* A, const double* V, double* Out,
                          cudaStream_t s)
{
    if (nblocks > 0) b_gemm<<<nblocks, 128, 0, s>>>(pr, np, nblocks, A, V, Out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_b_residual(const BProb* pr, int np, int nblocks, const double* X, const double* lam, double* R,
                              double* part, double* res, cudaStream_t s)
{
    if (nblocks > 0) b_residual<<<nblocks, 256, 0, s>>>(pr, np, nblocks, X, lam, R, part);
    b_residual_cols<<<dim3(1, np), 128, 0, s>>>(pr, part, res);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_b_reduced(const BProb* pr, int np, const double* Aq, const double* Bq, double* lam, double* V,
                             int* mk, double* work, cudaStream_t s)
{
    b_reduced<<<np, kRedThreads, 0, s>>>(pr, Aq, Bq, lam, V, mk, work);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace feast
