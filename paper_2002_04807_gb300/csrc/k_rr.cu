// Rayleigh-Ritz kernels, all FP64 (FEAST v4.0 guide Sec. 1.1: the reduced
// problem is built from the filtered subspace; Sec. 3.2: residuals
// ||A x - lambda B x|| / ||alpha B x||, alpha = max(|Emin|, |Emax|)).
//
// Blocks of vectors are row-major n x m (each row's m values contiguous), so a
// warp reads one matrix row of a block as one contiguous segment and the
// tall-skinny contractions stream rows.
//
//   spmm_f64      Y = A X                      (warp per row, shuffled indices)
//   gram_f64      C = X^T Y (m x m), split-K over rows, FP64 tensor cores
//                 (mma.sync m8n8k4 f64), upper tile triangle only, then a
//                 fixed-order reduction that mirrors the triangle
//   gemm_nn_f64   C = A V  (n x m times m x k), same tensor-core tile
//   residual_f64  R = A X - B X diag(lambda) and per-column ||R_j||, ||B x_j||
#include <atomic>

#include "feast_internal.cuh"

namespace feast {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launches(int k) { g_launches += k; }

// SM count of the device current at the first call (initialised once,
// thread-safe; every GPU of a process is assumed to be the same part).
int num_sms()
{
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

// ---------------------------------------------------------------- SpMM (real, FP64)
__global__ void __launch_bounds__(256) spmm_f64(int n, int m, const int* __restrict__ ia,
                                                const int* __restrict__ ja, const double* __restrict__ av,
                                                const double* __restrict__ X, double* __restrict__ Y)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nwarps) {
        const int s = __ldg(ia + i), e = __ldg(ia + i + 1);
        for (int c0 = 0; c0 < m; c0 += 32) {
            const int c = c0 + lane;
            double acc = 0.0;
            for (int base = s; base < e; base += 32) {
                const int cnt = min(32, e - base);
                int jl = 0;
                double al = 0.0;
                if (lane < cnt) {
                    jl = __ldg(ja + base + lane);
                    al = __ldg(av + base + lane);
                }
                for (int t = 0; t < cnt; ++t) {
                    const int j = __shfl_sync(0xffffffffu, jl, t);
                    const double a = __shfl_sync(0xffffffffu, al, t);
                    if (c < m) acc = fma(a, __ldg(X + (size_t)j * m + c), acc);
                }
            }
            if (c < m) Y[(size_t)i * m + c] = acc;
        }
    }
}

cudaError_t launch_spmm_f64(int n, int m, const int* ia, const int* ja, const double* av, const double* X,
                            double* Y, cudaStream_t s)
{
    if (n <= 0 || m <= 0) return cudaSuccess;
    long long blocks = ((long long)n + 7) / 8;
    const long long cap = (long long)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    spmm_f64<<<(int)blocks, 256, 0, s>>>(n, m, ia, ja, av, X, Y);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 tensor-core tile
// 64 x 64 output tile per CTA of 128 threads (2 x 2 warps of 32 x 32); K staged
// 16 at a time.  Shared tiles are K-major: As[k][r], Bs[k][c], leading
// dimension 68 so the 16 lanes of each half-warp hit distinct banks.
static constexpr int TM = 64, TK = 16, TLD = TM + 4;

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

__device__ __forceinline__ void tile_mma(const double (*As)[TLD], const double (*Bs)[TLD], double (&acc)[4][4][2],
                                         int wr, int wc, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < TK; kk += 4) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk + t][wr + i * 8 + g];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk + t][wc + j * 8 + g];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], a[i], b[j]);
    }
}

// Partial C tile (rows a0.., cols b0..) = sum over rows r in [r0, r1) of X[r][a] Y[r][b].
__global__ void __launch_bounds__(128) gram_f64(int n, int m, const double* __restrict__ X,
                                                const double* __restrict__ Y, double* __restrict__ part,
                                                int ksplit, int ntile)
{
    __shared__ __align__(16) double As[TK][TLD];
    __shared__ __align__(16) double Bs[TK][TLD];
    // upper-triangular tile index -> (ta, tb), ta <= tb
    int t = blockIdx.x, ta = 0;
    while (t >= ntile - ta) { t -= ntile - ta; ++ta; }
    const int tb = ta + t;
    const int a0 = ta * TM, b0 = tb * TM;
    const int split = blockIdx.y;
    const long long chunk = ((long long)n + ksplit - 1) / ksplit;
    const int r0 = (int)min((long long)n, split * chunk), r1 = (int)min((long long)n, (split + 1) * chunk);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    // a warp's 32 x 32 sub-tile is needed when it lies inside the m x m matrix
    // and is not strictly below the diagonal (the result keeps the upper
    // triangle); the others only help load the shared tiles
    const bool live = a0 + wr < m && b0 + wc < m && !(ta == tb && wr > wc);
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    for (int k0 = r0; k0 < r1; k0 += TK) {
        // 16 rows x 64 cols for each operand: 1024 values, 8 per thread
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int idx = tid + q * 128;
            const int kk = idx >> 6, c = idx & 63;
            const int r = k0 + kk;
            const bool rok = r < r1;
            As[kk][c] = (rok && a0 + c < m) ? __ldg(X + (size_t)r * m + a0 + c) : 0.0;
            Bs[kk][c] = (rok && b0 + c < m) ? __ldg(Y + (size_t)r * m + b0 + c) : 0.0;
        }
        __syncthreads();
        if (live) tile_mma(As, Bs, acc, wr, wc, lane);  // warp-uniform
        __syncthreads();
    }
    if (!live) return;
    double* out = part + (size_t)split * m * m;
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

// C[i][j] = the upper-triangle partial at (min(i,j), max(i,j)), summed over
// splits in order: the upper triangle of X^T Y, mirrored.
__global__ void gram_reduce(int m, const double* __restrict__ part, int ksplit, double* __restrict__ C)
{
    const long long total = (long long)m * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / m), j = (int)(idx % m);
        const int a = i < j ? i : j, b = i < j ? j : i;
        double v = 0.0;
        for (int s = 0; s < ksplit; ++s) v += part[(size_t)s * m * m + (size_t)a * m + b];
        C[idx] = v;
    }
}

size_t gram_partial_doubles(int n, int m, int* ksplit_out, int nsm)
{
    const int nt = (m + TM - 1) / TM;
    const int tiles = nt * (nt + 1) / 2;
    int ks = (4 * nsm + tiles - 1) / tiles;
    const int maxk = (n + 255) / 256;  // at least 256 rows per split
    if (ks > maxk) ks = maxk;
    if (ks < 1) ks = 1;
    if (ksplit_out) *ksplit_out = ks;
    return (size_t)ks * m * m;
}

cudaError_t launch_gram_reduce(int m, const double* part, int ksplit, double* C, cudaStream_t s)
{
    long long blocks = ((long long)m * m + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    gram_reduce<<<(int)blocks, 256, 0, s>>>(m, part, ksplit, C);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gram_f64(int n, int m, const double* X, const double* Y, double* C, double* part, int ksplit,
                            int sym, cudaStream_t s)
{
    (void)sym;
    if (m <= 0) return cudaSuccess;
    const int nt = (m + TM - 1) / TM;
    dim3 grid(nt * (nt + 1) / 2, ksplit);
    gram_f64<<<grid, 128, 0, s>>>(n, m, X, Y, part, ksplit, nt);
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long blocks = ((long long)m * m + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    gram_reduce<<<(int)blocks, 256, 0, s>>>(m, part, ksplit, C);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- C = A V
__global__ void __launch_bounds__(128) gemm_nn_f64(int n, int m, int k, const double* __restrict__ A,
                                                   const double* __restrict__ V, double* __restrict__ C)
{
    __shared__ __align__(16) double As[TK][TLD];
    __shared__ __align__(16) double Bs[TK][TLD];
    const int r0 = blockIdx.x * TM, c0 = blockIdx.y * TM;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    for (int k0 = 0; k0 < m; k0 += TK) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int idx = tid + q * 128;
            // A tile: 64 rows x 16 k, row-major in global -> transposed into As[k][row]
            const int ar = idx >> 4, ak = idx & 15;
            const int gr = r0 + ar, gk = k0 + ak;
            As[ak][ar] = (gr < n && gk < m) ? __ldg(A + (size_t)gr * m + gk) : 0.0;
            // V tile: 16 k x 64 cols
            const int bk = idx >> 6, bc = idx & 63;
            const int vk = k0 + bk, vc = c0 + bc;
            Bs[bk][bc] = (vk < m && vc < k) ? __ldg(V + (size_t)vk * k + vc) : 0.0;
        }
        __syncthreads();
        tile_mma(As, Bs, acc, wr, wc, lane);
        __syncthreads();
    }
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int row = r0 + wr + i * 8 + g;
            const int col = c0 + wc + j * 8 + 2 * tq;
            if (row < n && col < k) C[(size_t)row * k + col] = acc[i][j][0];
            if (row < n && col + 1 < k) C[(size_t)row * k + col + 1] = acc[i][j][1];
        }
}

cudaError_t launch_gemm_nn_f64(int n, int m, int k, const double* A, const double* V, double* C, cudaStream_t s)
{
    if (n <= 0 || k <= 0) return cudaSuccess;
    dim3 grid((n + TM - 1) / TM, (k + TM - 1) / TM);
    gemm_nn_f64<<<grid, 128, 0, s>>>(n, m, k, A, V, C);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- residuals
// Pass 1: per row block (RR_RB rows), R rows and per-column partial sums of
// R^2 and (Bx)^2 -> part[rb][m][2].  Pass 2: fixed-order column sums.
static constexpr int RR_RB = 256;

__global__ void __launch_bounds__(256) residual_rows(int n, int m, const int* __restrict__ ia,
                                                     const int* __restrict__ ja, const double* __restrict__ av,
                                                     const int* __restrict__ ib, const int* __restrict__ jb,
                                                     const double* __restrict__ bv, const double* __restrict__ X,
                                                     const double* __restrict__ lam, double* __restrict__ R,
                                                     double* __restrict__ part)
{
    __shared__ double sr[8][32];
    __shared__ double sb[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nrb = (n + RR_RB - 1) / RR_RB;
    const int nchunk = (m + 31) / 32;
    for (int it = blockIdx.x; it < nrb * nchunk; it += gridDim.x) {
        const int rb = it / nchunk, ch = it % nchunk;
        const int c = ch * 32 + lane;
        const double l = c < m ? lam[c] : 0.0;
        double accr = 0.0, accb = 0.0;
        for (int i = rb * RR_RB + warp; i < min(n, (rb + 1) * RR_RB); i += 8) {
            double ax = 0.0, bx = 0.0;
            {
                const int s = __ldg(ia + i), e = __ldg(ia + i + 1);
                for (int base = s; base < e; base += 32) {
                    const int cnt = min(32, e - base);
                    int jl = 0;
                    double al = 0.0;
                    if (lane < cnt) { jl = __ldg(ja + base + lane); al = __ldg(av + base + lane); }
                    for (int t = 0; t < cnt; ++t) {
                        const int j = __shfl_sync(0xffffffffu, jl, t);
                        const double a = __shfl_sync(0xffffffffu, al, t);
                        if (c < m) ax = fma(a, __ldg(X + (size_t)j * m + c), ax);
                    }
                }
            }
            if (ib == nullptr) {
                if (c < m) bx = __ldg(X + (size_t)i * m + c);
            } else {
                const int s = __ldg(ib + i), e = __ldg(ib + i + 1);
                for (int base = s; base < e; base += 32) {
                    const int cnt = min(32, e - base);
                    int jl = 0;
                    double al = 0.0;
                    if (lane < cnt) { jl = __ldg(jb + base + lane); al = __ldg(bv + base + lane); }
                    for (int t = 0; t < cnt; ++t) {
                        const int j = __shfl_sync(0xffffffffu, jl, t);
                        const double a = __shfl_sync(0xffffffffu, al, t);
                        if (c < m) bx = fma(a, __ldg(X + (size_t)j * m + c), bx);
                    }
                }
            }
            if (c < m) {
                const double r = fma(-l, bx, ax);
                R[(size_t)i * m + c] = r;
                accr = fma(r, r, accr);
                accb = fma(bx, bx, accb);
            }
        }
        sr[warp][lane] = accr;
        sb[warp][lane] = accb;
        __syncthreads();
        if (warp == 0 && c < m) {
            double s1 = 0.0, s2 = 0.0;
            for (int w = 0; w < 8; ++w) { s1 += sr[w][lane]; s2 += sb[w][lane]; }
            part[((size_t)rb * m + c) * 2] = s1;
            part[((size_t)rb * m + c) * 2 + 1] = s2;
        }
        __syncthreads();
    }
}

__global__ void residual_cols(int n, int m, const double* __restrict__ part, double alpha, double* __restrict__ res,
                              double* __restrict__ rnorm)
{
    const int nrb = (n + RR_RB - 1) / RR_RB;
    const int c = blockIdx.x;
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (int rb = threadIdx.x; rb < nrb; rb += blockDim.x) {
        a += part[((size_t)rb * m + c) * 2];
        b += part[((size_t)rb * m + c) * 2 + 1];
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
        if (rnorm) rnorm[c] = rn;
    }
}

size_t residual_partial_doubles(int n, int m)
{
    return (size_t)((n + RR_RB - 1) / RR_RB) * m * 2;
}

cudaError_t launch_residual_f64(int n, int m, const int* ia, const int* ja, const double* av, const int* ib,
                                const int* jb, const double* bv, const double* X, const double* lam, double* R,
                                double* part, unsigned* counter, double* res, double alpha, cudaStream_t s)
{
    (void)counter;
    if (n <= 0 || m <= 0) return cudaSuccess;
    const int nrb = (n + RR_RB - 1) / RR_RB, nchunk = (m + 31) / 32;
    long long items = (long long)nrb * nchunk;
    long long cap = (long long)num_sms() * 8;
    int grid = (int)(items < cap ? items : cap);
    residual_rows<<<grid, 256, 0, s>>>(n, m, ia, ja, av, ib, jb, bv, X, lam, R, part);
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    residual_cols<<<m, 256, 0, s>>>(n, m, part, alpha, res, nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- column dots
// t[c] = sum_i X[i][c] Y[i][c] over row-major n x m blocks (the probe terms
// y_c^T Q_c of the stochastic eigenvalue count).  Pass 1: per row block of
// RR_RB rows, one warp-row sweep per 32 columns, fixed-order partials
// part[rb][c]; pass 2: fixed-order sum over the row blocks.
__global__ void __launch_bounds__(256) coldot_rows(int n, int m, const double* __restrict__ X,
                                                   const double* __restrict__ Y, double* __restrict__ part)
{
    __shared__ double sh[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nrb = (n + RR_RB - 1) / RR_RB;
    const int nchunk = (m + 31) / 32;
    for (int it = blockIdx.x; it < nrb * nchunk; it += gridDim.x) {
        const int rb = it / nchunk, ch = it % nchunk;
        const int c = ch * 32 + lane;
        double acc = 0.0;
        if (c < m)
            for (int i = rb * RR_RB + warp; i < min(n, (rb + 1) * RR_RB); i += 8)
                acc = fma(X[(size_t)i * m + c], Y[(size_t)i * m + c], acc);
        sh[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && c < m) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += sh[w][lane];
            part[(size_t)rb * m + c] = t;
        }
        __syncthreads();
    }
}

__global__ void coldot_cols(int n, int m, const double* __restrict__ part, double* __restrict__ t)
{
    const int nrb = (n + RR_RB - 1) / RR_RB;
    const int c = blockIdx.x;
    __shared__ double sh[256];
    double a = 0.0;
    for (int rb = threadIdx.x; rb < nrb; rb += blockDim.x) a += part[(size_t)rb * m + c];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) t[c] = sh[0];
}

// part: at least residual_partial_doubles(n, m) / 2 doubles.
cudaError_t launch_coldot_f64(int n, int m, const double* X, const double* Y, double* part, double* t, cudaStream_t s)
{
    if (n <= 0 || m <= 0) return cudaSuccess;
    const long long items = (long long)((n + RR_RB - 1) / RR_RB) * ((m + 31) / 32);
    const long long cap = (long long)num_sms() * 8;
    coldot_rows<<<(int)(items < cap ? items : cap), 256, 0, s>>>(n, m, X, Y, part);
    coldot_cols<<<m, 256, 0, s>>>(n, m, part, t);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace feast
