// FP64-accurate Gram contraction C = X^T Y on the BF16 tensor cores, for the
// Rayleigh-Ritz projections A_Q = Q^T (A Q) and B_Q = Q^T (B Q) (FEAST v4.0
// guide, Sec. 1.1: the reduced problem of the filtered subspace, in FP64).
//
// GB300 keeps little FP64 tensor throughput, so the projection is rebuilt from
// exact integer products, after the splitting scheme of Ozaki, Ogita, Oishi
// and Rump ("Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication", 2012):
//   * every column c of X (of Y) gets a power of two 2^E_c > max_i |X[i][c]|;
//   * |X[i][c]| 2^-E_c lies in [0, 1) and is written with kSlices base-2^7
//     digits, |x| 2^-E = sum_s d_s 2^(-7 s) + r, d_s in [0, 127] (with the
//     sign of x), 0 <= r < 2^(-7 kSlices); the digits come from the FP64 bit
//     pattern by integer shifts and are exact in BF16;
//   * X[i][a] Y[i][b] = 2^(E_a + F_b) sum_{s,t} d_s(i,a) e_t(i,b) 2^(-7 (s+t)),
//     the pairs with s + t <= kSlices + 1 are kept (the rest weigh below
//     2^(-7 kSlices) relative to 2^(E_a + F_b));
//   * a level L = s + t has at most kSlices pairs of products below 2^14, so
//     its sum over 128 rows stays below 2^24 and mma.sync accumulates it in
//     FP32 without any rounding; every 128 rows the level sums are folded,
//     exactly, into two 64-bit integer accumulators (oz_fold), and at the end
//     they are turned into FP64 once and the column scales 2^(E_a + F_b) are
//     applied.
// With kSlices = 8 the kept part is exact and the truncation error of an
// element is below 2^-55 |2^E_a| |2^F_b| per row: at FP64 level.
//
// Layout: X, Y row-major n x m FP64.  A CTA (four warps) owns one 32 x 32
// output tile of the upper tile triangle and a range of rows (split-K); each
// warp owns a 16 x 16 quarter.  Per chunk of 32 rows the CTA loads the tile's
// 32 columns of X and of Y, cuts them into slices and stores the slices in
// shared memory as BF16 pairs of consecutive rows (the k-pairs of an mma
// fragment), [slice][k-pair][column] with a row stride of 40 words so the
// fragment loads of a warp hit distinct banks.  Three CTAs per SM overlap one
// CTA's loads and cuts with another's tensor-core work.
// Partial tiles go to the split-K buffer and gram_reduce (k_rr.cu) sums them
// in a fixed order and mirrors the upper triangle.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "feast_internal.cuh"

namespace feast {

static constexpr int kSlices = 8;
static constexpr int kOzTile = 32;                  // output tile side (CTA)
static constexpr int kOzChunk = 32;                 // rows per shared-memory chunk
static constexpr int kOzFlushChunks = 4;            // chunks per FP32 -> FP64 flush (128 rows)
static constexpr int kOzStride = 40;                // words per k-pair row in shared memory
static constexpr int kOzPlane = (kOzChunk / 2) * kOzStride;  // words per slice plane
static constexpr int kOzThreads = 128;

// ---------------------------------------------------------------- column exponents
// ex[c] = max over rows of the biased FP64 exponent field of |X[i][c]| (0 for
// a zero column); |X[i][c]| < 2^(ex[c] - 1022).  ex must be zeroed first.
__global__ void __launch_bounds__(256) oz_colexp(int n, int m, const double* __restrict__ X, int* __restrict__ ex)
{
    const int rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        int e = 0;
        for (int r = r0; r < r1; ++r) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(__ldg(X + (size_t)r * m + c));
            e = max(e, (int)((b >> 52) & 0x7ff));
        }
        if (e > 0) atomicMax(ex + c, e);
    }
}

// E_c of the splitting from the exponent field: |x| < 2^E_c, clamped so that
// 2^-E_c is a normal double.
__device__ __forceinline__ int oz_scale_exp(int field) { return min(max(field - 1022, -1022), 1022); }

// The kSlices base-2^7 digits of |x| 2^-E, most significant first, with the
// sign of x, by integer operations on the FP64 bit pattern (GB300's FP64 ALU
// is too slow for the cut): |x| = M 2^(e - 1075) with M the 53-bit
// significand, and F = floor(|x| 2^(56 - E)) = M 2^(e - 1075 - E + 56) < 2^56
// because |x| < 2^E; then |x| 2^-E = sum_s d_s 2^(-7 (s + 1)) + r with
// 0 <= r < 2^-56, d_s in [0, 127].
__device__ __forceinline__ void oz_cut(double x, int E, float (&d)[kSlices])
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7ff);
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
    const int sh = (ef ? ef : 1) - 1075 - E + 56;  // <= 3 for |x| < 2^E
    const unsigned long long F = sh >= 0 ? (M << min(sh, 3)) : (sh > -64 ? (M >> -sh) : 0ull);
    const float sg = (b >> 63) ? -1.f : 1.f;
#pragma unroll
    for (int s = 0; s < kSlices; ++s) d[s] = sg * (float)(unsigned)((F >> (49 - 7 * s)) & 127ull);
}

// Exact folding of the FP32 level sums into two 64-bit integer accumulators.
// Level l (weight 2^(-7 (l + 2))) holds an integer below 2^24, so
//   hi = sum_{l < 4} P_l 2^(7 (3 - l))   in units of 2^-35,
//   lo = sum_{l >= 4} P_l 2^(7 (7 - l))  in units of 2^-63,
// are below 2^46 per flush and exact, and so are their running sums (below
// 2^63 for up to 2^17 flushes).  FP64 (scarce on GB300) is used only once per
// element at the end: value = hi 2^-35 + lo 2^-63.
__device__ __forceinline__ void oz_fold(float (&P)[kSlices], long long& hi, long long& lo)
{
    long long h = 0, l = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) h += (long long)__float2int_rn(P[s]) * (1LL << (7 * (3 - s)));
#pragma unroll
    for (int s = 4; s < kSlices; ++s) l += (long long)__float2int_rn(P[s]) * (1LL << (7 * (7 - s)));
    hi += h;
    lo += l;
}

__device__ __forceinline__ double oz_value(long long hi, long long lo, int e)
{
    return ldexp(fma((double)hi, 0x1p-35, (double)lo * 0x1p-63), e);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Partial C tile (rows a0.., cols b0..) of X^T Y over rows [r0, r1).
__global__ void __launch_bounds__(kOzThreads, 3) gram_oz(int n, int m, const double* __restrict__ X,
                                                           const double* __restrict__ Y, const int* __restrict__ exX,
                                                           const int* __restrict__ exY, double* __restrict__ part,
                                                           int ksplit, int ntile, long long rows_per_split, int full)
{
    __shared__ uint32_t sA[kSlices * kOzPlane];
    __shared__ uint32_t sB[kSlices * kOzPlane];
    int ta = 0, tb = 0;
    if (full) {  // every tile (X^T Y need not be symmetric)
        ta = blockIdx.x / ntile;
        tb = blockIdx.x % ntile;
    } else {  // upper tile triangle
        int t = blockIdx.x;
        while (t >= ntile - ta) { t -= ntile - ta; ++ta; }
        tb = ta + t;
    }
    const int a0 = ta * kOzTile, b0 = tb * kOzTile;
    const int split = blockIdx.y;
    const int r0 = (int)min((long long)n, split * rows_per_split);
    const int r1 = (int)min((long long)n, (split + 1) * rows_per_split);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 16, wc = (warp & 1) * 16;
    const int g = lane >> 2, tq = lane & 3;
    // a warp's 16 x 16 quarter is needed when it lies inside the m x m matrix
    // and not strictly below the diagonal; the others only help with loads
    const bool live = a0 + wr < m && b0 + wc < m && (full || !(ta == tb && wr > wc));

    // loader: thread owns column lane of the tile and k-pairs warp + 4 u
    const int ca = a0 + lane, cb = b0 + lane;
    const int Ex = (ca < m) ? oz_scale_exp(__ldg(exX + ca)) : 0;
    const int Ey = (cb < m) ? oz_scale_exp(__ldg(exY + cb)) : 0;
    double vx[8], vy[8];  // [u][row of the pair]
    auto load = [&](int rbase) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = rbase + 2 * (warp + 4 * u) + h;
                const bool ok = r < r1;
                vx[2 * u + h] = (ok && ca < m) ? __ldg(X + (size_t)r * m + ca) : 0.0;
                vy[2 * u + h] = (ok && cb < m) ? __ldg(Y + (size_t)r * m + cb) : 0.0;
            }
        }
    };

    float acc[kSlices][2][4];
#pragma unroll
    for (int l = 0; l < kSlices; ++l)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[l][j][q] = 0.f;
    long long ahi[2][4], alo[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) ahi[j][q] = alo[j][q] = 0;

    auto flush = [&]() {
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float P[kSlices];
#pragma unroll
                for (int l = 0; l < kSlices; ++l) {
                    P[l] = acc[l][j][q];
                    acc[l][j][q] = 0.f;
                }
                oz_fold(P, ahi[j][q], alo[j][q]);
            }
    };

    int nchunk = 0;
    for (int rbase = r0; rbase < r1; rbase += kOzChunk) {
        load(rbase);
        __syncthreads();  // the previous chunk's fragments have been read
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float dx0[kSlices], dx1[kSlices], dy0[kSlices], dy1[kSlices];
            oz_cut(vx[2 * u], Ex, dx0);
            oz_cut(vx[2 * u + 1], Ex, dx1);
            oz_cut(vy[2 * u], Ey, dy0);
            oz_cut(vy[2 * u + 1], Ey, dy1);
            const int w = (warp + 4 * u) * kOzStride + lane;
#pragma unroll
            for (int s = 0; s < kSlices; ++s) {
                sA[s * kOzPlane + w] = pack_bf16x2(dx0[s], dx1[s]);
                sB[s * kOzPlane + w] = pack_bf16x2(dy0[s], dy1[s]);
            }
        }
        __syncthreads();
        if (live) {  // warp-uniform
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const int j0 = kk * 8 + tq;
                uint32_t bf[kSlices][2][2];
#pragma unroll
                for (int s = 0; s < kSlices; ++s)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        const int col = wc + nt * 8 + g;
                        bf[s][nt][0] = sB[s * kOzPlane + j0 * kOzStride + col];
                        bf[s][nt][1] = sB[s * kOzPlane + (j0 + 4) * kOzStride + col];
                    }
#pragma unroll
                for (int s = 0; s < kSlices; ++s) {
                    const uint32_t* pa = sA + s * kOzPlane;
                    const uint32_t fa0 = pa[j0 * kOzStride + wr + g];
                    const uint32_t fa1 = pa[j0 * kOzStride + wr + g + 8];
                    const uint32_t fa2 = pa[(j0 + 4) * kOzStride + wr + g];
                    const uint32_t fa3 = pa[(j0 + 4) * kOzStride + wr + g + 8];
#pragma unroll
                    for (int t2 = 0; t2 < kSlices - s; ++t2)
#pragma unroll
                        for (int nt = 0; nt < 2; ++nt)
                            mma_bf16(acc[s + t2][nt], fa0, fa1, fa2, fa3, bf[t2][nt][0], bf[t2][nt][1]);
                }
            }
        }
        if (++nchunk == kOzFlushChunks) {
            flush();
            nchunk = 0;
        }
    }
    flush();
    if (!live) return;
    double* out = part + (size_t)split * m * m;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = a0 + wr + g + (q >= 2 ? 8 : 0);
            const int col = b0 + wc + nt * 8 + 2 * tq + (q & 1);
            if (row < m && col < m) {
                const int e = oz_scale_exp(__ldg(exX + row)) + oz_scale_exp(__ldg(exY + col));
                out[(size_t)row * m + col] = oz_value(ahi[nt][q], alo[nt][q], e);
            }
        }
}

// C[i][j] = sum over splits of part[s][i][j], in split order (full product).
__global__ void gram_reduce_full(int m, const double* __restrict__ part, int ksplit, double* __restrict__ C)
{
    const long long total = (long long)m * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < ksplit; ++s) v += part[(size_t)s * total + idx];
        C[idx] = v;
    }
}

size_t gram_oz_partial_doubles(int n, int m, int* ksplit_out, long long* rows_per_split, int nsm, bool full)
{
    const int nt = (m + kOzTile - 1) / kOzTile;
    const int tiles = full ? nt * nt : nt * (nt + 1) / 2;
    int ks = (3 * nsm) / tiles;  // one wave of three CTAs per SM
    const int maxk = (n + 255) / 256;        // at least 256 rows per split
    if (ks > maxk) ks = maxk;
    if (ks < 1) ks = 1;
    long long rps = ((long long)n + ks - 1) / ks;
    rps = (rps + kOzChunk - 1) / kOzChunk * kOzChunk;  // whole chunks
    ks = (int)(((long long)n + rps - 1) / rps);
    if (ks < 1) ks = 1;
    if (ksplit_out) *ksplit_out = ks;
    if (rows_per_split) *rows_per_split = rps;
    return (size_t)ks * m * m;
}

size_t gram_oz_work_bytes(int m) { return (size_t)2 * m * sizeof(int) + 256; }

cudaError_t launch_gram_oz(int n, int m, const double* X, const double* Y, double* C, double* part, int* ex,
                           cudaStream_t s, bool full)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    int ks = 1;
    long long rps = 0;
    gram_oz_partial_doubles(n, m, &ks, &rps, num_sms(), full);
    int* exX = ex;
    int* exY = ex + m;
    cudaError_t e = cudaMemsetAsync(ex, 0, sizeof(int) * 2 * (size_t)m, s);
    if (e != cudaSuccess) return e;
    int blocks = (int)std::min<long long>(((long long)n + 127) / 128, (long long)num_sms() * 4);
    if (blocks < 1) blocks = 1;
    oz_colexp<<<blocks, 256, 0, s>>>(n, m, X, exX);
    if (Y != X) oz_colexp<<<blocks, 256, 0, s>>>(n, m, Y, exY);
    else if ((e = cudaMemcpyAsync(exY, exX, sizeof(int) * m, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    const int nt = (m + kOzTile - 1) / kOzTile;
    dim3 grid(full ? nt * nt : nt * (nt + 1) / 2, ks);
    gram_oz<<<grid, kOzThreads, 0, s>>>(n, m, X, Y, exX, exY, part, ks, nt, rps, full ? 1 : 0);
    count_launches(Y != X ? 4 : 3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!full) return launch_gram_reduce(m, part, ks, C, s);
    const int rblocks = (int)std::min<long long>(((long long)m * m + 255) / 256, 2048);
    gram_reduce_full<<<rblocks, 256, 0, s>>>(m, part, ks, C);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- C = A V
// The Ritz vectors X = Q V (A row-major n x m, V row-major m x k, C row-major
// n x k) by the same splitting, now along the contraction index of A's rows:
// row i of A gets its own power of two 2^E_i > max_a |A[i][a]|, column c of V
// its 2^F_c, so every product of a row slice and a column slice lies on one
// integer grid per output element.  V is cut once into slice planes
// Vs[slice][column][k-pair] (oz_split_cols); A's rows are cut by the CTAs
// that use them.  A level's sum over 128 contraction steps stays below 2^24
// (as for the Gram), so the FP32 level sums are folded into the integer
// accumulators every 128 steps of the contraction and scaled by 2^(E_i + F_c)
// at the end.

// ex[i] = largest biased exponent field over row i of the row-major n x m A.
__global__ void __launch_bounds__(256) oz_rowexp(int n, int m, const double* __restrict__ A, int* __restrict__ ex)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nw) {
        int e = 0;
        for (int a = lane; a < m; a += 32) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(__ldg(A + (size_t)i * m + a));
            e = max(e, (int)((b >> 52) & 0x7ff));
        }
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (lane == 0) ex[i] = e;
    }
}

// Vs[s][c][j] (c < kp, j < mp/2) = BF16 pair (d_s(V[2j][c]), d_s(V[2j+1][c]))
// under the column scale of c; zero outside m x k.
__global__ void oz_split_cols(int m, int k, int kp, int mp, const double* __restrict__ V, const int* __restrict__ exV,
                              uint32_t* __restrict__ Vs)
{
    const int half = mp / 2;
    const long long total = (long long)kp * half;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / half), j = (int)(t % half);
        float d0[kSlices], d1[kSlices];
        double v0 = 0.0, v1 = 0.0;
        int E = 0;
        if (c < k) {
            E = oz_scale_exp(exV[c]);
            if (2 * j < m) v0 = V[(size_t)(2 * j) * k + c];
            if (2 * j + 1 < m) v1 = V[(size_t)(2 * j + 1) * k + c];
        }
        oz_cut(v0, E, d0);
        oz_cut(v1, E, d1);
#pragma unroll
        for (int s = 0; s < kSlices; ++s) Vs[((size_t)s * kp + c) * half + j] = pack_bf16x2(d0[s], d1[s]);
    }
}

// One 32 x 32 tile of C per CTA (four warps of 16 x 16), contraction in
// chunks of 32.  Shared slices: A [slice][row][k-pair], V [slice][column][k-pair],
// 20 words per row (16 k-pairs + 4 of padding: conflict-free fragment loads).
static constexpr int kGzStride = 20;
static constexpr int kGzPlane = 32 * kGzStride;

__global__ void __launch_bounds__(kOzThreads, 3) gemm_oz(int n, int m, int k, int kp, int mp,
                                                           const double* __restrict__ A, const uint32_t* __restrict__ Vs,
                                                           const int* __restrict__ exA, const int* __restrict__ exV,
                                                           double* __restrict__ C)
{
    __shared__ uint32_t sA[kSlices * kGzPlane];
    __shared__ uint32_t sV[kSlices * kGzPlane];
    const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = (warp >> 1) * 16, wc = (warp & 1) * 16;
    const int g = lane >> 2, tq = lane & 3;
    const int half = mp / 2;
    // A loader: thread owns rows warp + 4 u (u < 8) of the tile and k-pair lane & 15,
    // lanes 16..31 the same k-pairs of the next row group
    float acc[kSlices][2][4];
#pragma unroll
    for (int l = 0; l < kSlices; ++l)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[l][j][q] = 0.f;
    long long ahi[2][4], alo[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) ahi[j][q] = alo[j][q] = 0;
    const int jl = lane & 15;
    int rs[4];  // scale exponents E of the loader's rows
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = i0 + warp * 8 + 2 * u + (lane >> 4);
        rs[u] = r < n ? oz_scale_exp(__ldg(exA + r)) : 0;
    }
    int nchunk = 0;
    for (int a0 = 0; a0 < mp; a0 += 32) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int rl = warp * 8 + 2 * u + (lane >> 4);  // row of the tile
            const int r = i0 + rl;
            const int a = a0 + 2 * jl;
            double v0 = 0.0, v1 = 0.0;
            if (r < n) {
                if (a < m) v0 = __ldg(A + (size_t)r * m + a);
                if (a + 1 < m) v1 = __ldg(A + (size_t)r * m + a + 1);
            }
            float d0[kSlices], d1[kSlices];
            oz_cut(v0, rs[u], d0);
            oz_cut(v1, rs[u], d1);
#pragma unroll
            for (int s = 0; s < kSlices; ++s) sA[s * kGzPlane + rl * kGzStride + jl] = pack_bf16x2(d0[s], d1[s]);
        }
        // V slices of this chunk: 32 columns x 16 k-pairs per slice
        for (int t = tid; t < kSlices * 32 * 16; t += kOzThreads) {
            const int s = t / 512, rem = t % 512, cl = rem / 16, j = rem % 16;
            sV[s * kGzPlane + cl * kGzStride + j] = __ldg(Vs + ((size_t)s * kp + c0 + cl) * half + a0 / 2 + j);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int j0 = kk * 8 + tq;
            uint32_t bf[kSlices][2][2];
#pragma unroll
            for (int s = 0; s < kSlices; ++s)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const int col = wc + nt * 8 + g;
                    bf[s][nt][0] = sV[s * kGzPlane + col * kGzStride + j0];
                    bf[s][nt][1] = sV[s * kGzPlane + col * kGzStride + j0 + 4];
                }
#pragma unroll
            for (int s = 0; s < kSlices; ++s) {
                const uint32_t* pa = sA + s * kGzPlane;
                const uint32_t fa0 = pa[(wr + g) * kGzStride + j0];
                const uint32_t fa1 = pa[(wr + g + 8) * kGzStride + j0];
                const uint32_t fa2 = pa[(wr + g) * kGzStride + j0 + 4];
                const uint32_t fa3 = pa[(wr + g + 8) * kGzStride + j0 + 4];
#pragma unroll
                for (int t2 = 0; t2 < kSlices - s; ++t2)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
                        mma_bf16(acc[s + t2][nt], fa0, fa1, fa2, fa3, bf[t2][nt][0], bf[t2][nt][1]);
            }
        }
        if (++nchunk == kOzFlushChunks || a0 + 32 >= mp) {
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float P[kSlices];
#pragma unroll
                    for (int l = 0; l < kSlices; ++l) {
                        P[l] = acc[l][j][q];
                        acc[l][j][q] = 0.f;
                    }
                    oz_fold(P, ahi[j][q], alo[j][q]);
                }
            nchunk = 0;
        }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = i0 + wr + g + (q >= 2 ? 8 : 0);
            const int col = c0 + wc + nt * 8 + 2 * tq + (q & 1);
            if (row < n && col < k) {
                const int e = oz_scale_exp(__ldg(exA + row)) + oz_scale_exp(__ldg(exV + col));
                C[(size_t)row * k + col] = oz_value(ahi[nt][q], alo[nt][q], e);
            }
        }
}

size_t gemm_oz_work_bytes(int n, int m, int k)
{
    const size_t kp = (size_t)(k + 31) / 32 * 32, mp = (size_t)(m + 31) / 32 * 32;
    return ((size_t)n + k) * sizeof(int) + 256 + kSlices * kp * (mp / 2) * sizeof(uint32_t) + 256;
}

cudaError_t launch_gemm_oz(int n, int m, int k, const double* A, const double* V, double* C, void* work,
                           cudaStream_t s)
{
    if (n <= 0 || k <= 0 || m <= 0) return cudaSuccess;
    const int kp = (k + 31) / 32 * 32, mp = (m + 31) / 32 * 32;
    char* p = (char*)work;
    int* exA = (int*)p;
    int* exV = exA + n;
    p += (((size_t)n + k) * sizeof(int) + 255) / 256 * 256;
    uint32_t* Vs = (uint32_t*)p;
    cudaError_t e = cudaMemsetAsync(exV, 0, sizeof(int) * (size_t)k, s);
    if (e != cudaSuccess) return e;
    int blocks = (int)std::min<long long>(((long long)n + 7) / 8, (long long)num_sms() * 8);
    oz_rowexp<<<blocks, 256, 0, s>>>(n, m, A, exA);
    oz_colexp<<<std::max(1, std::min(m, 64)), 256, 0, s>>>(m, k, V, exV);
    const long long sv = (long long)kp * (mp / 2);
    oz_split_cols<<<(int)std::min<long long>((sv + 255) / 256, 1024), 256, 0, s>>>(m, k, kp, mp, V, exV, Vs);
    dim3 grid((n + 31) / 32, kp / 32);
    gemm_oz<<<grid, kOzThreads, 0, s>>>(n, m, k, kp, mp, A, Vs, exA, exV, C);
    count_launches(4);
    return cudaGetLastError();
}

}  // namespace feast
