// FEAST driver for complex Hermitian CSR problems (FEAST v4.0 guide,
// Sec. 3.2 "FEAST Hermitian", zfeast_hcsr{ev,gv}; the algorithm of Sec. 1.1).
//
// The loop is the one of the real symmetric driver: a first contour pass on a
// start block (or Rayleigh-Ritz on a given subspace, fpm(5) = 1), then
// Rayleigh-Ritz, residuals, convergence test (fpm(6): residual or trace), and
// residual-inverse passes Q = X rho(Lambda) + sum_e (1/2)[c_e y_e + conj(c_e)
// yh_e].  The contour pass solves both halves of the contour by BiCG on
// z_e B - A with its conjugate-shift shadow system (k_herm.cu).  Complex
// blocks on the device are row-major n x m double2; the caller's X is
// column-major n x m0 complex (interleaved real, imaginary doubles).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/feast_gb300.h"
#include "feast_internal.cuh"
#include "herm_internal.cuh"

namespace feast {
int fpm_check(const int* fpm);
void contour_nodes(int rule, int ne, double emin, double emax, double ratio, std::vector<double>& zw);
int cuda_error(cudaError_t e, const char* where);
void clear_last_error();
void feast_log(int lvl, const char* text);
const char* set_last_error(const char* msg);
}  // namespace feast

using namespace feast;
using namespace feast::herm;

namespace {

#define HCK(x)                                              \
    do {                                                    \
        cudaError_t _e = (x);                               \
        if (_e != cudaSuccess) return cuda_error(_e, #x);   \
    } while (0)

int grid_of(long long total)
{
    long long b = (total + 255) / 256;
    const long long cap = (long long)num_sms() * 16;
    if (b > cap) b = cap;
    return (int)(b > 0 ? b : 1);
}

// Start block: uniform [-1, 1) real and imaginary parts from a counter-based
// hash (SplitMix64 finaliser) of (seed, index).
__device__ __forceinline__ double hash_unit(unsigned long long x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void hk_random(long long total, unsigned long long seed, double2* __restrict__ Y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        Y[i] = make_double2(hash_unit(seed * 0x100000001B3ull + 2 * i), hash_unit(seed * 0x100000001B3ull + 2 * i + 1));
}

// column-major n x m (caller layout) -> row-major
__global__ void hk_col_to_row(int n, int m, const double2* __restrict__ Xc, double2* __restrict__ Xr)
{
    const long long total = (long long)n * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / m, j = idx % m;
        Xr[idx] = Xc[j * n + i];
    }
}

// out[:, c] (column-major) = X[:, perm[c]] (row-major) for c < mk, zero for mk <= c < m
__global__ void hk_gather_cols(int n, int m, int mk, const double2* __restrict__ X, const int* __restrict__ perm,
                               double2* __restrict__ out)
{
    const long long total = (long long)n * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long c = idx / n, i = idx % n;
        out[idx] = c < mk ? X[i * m + perm[c]] : make_double2(0.0, 0.0);
    }
}

}  // namespace

namespace {

struct HDevMem {
    std::vector<void*> ptrs;
    ~HDevMem()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t count)
    {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T) + 256);
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            *p = (T*)q;
        }
        return e;
    }
};

struct HMat {
    int n = 0, nnz = 0;
    const int* ia = nullptr;
    const int* ja = nullptr;
    const double2* v = nullptr;  // FP64 values (Rayleigh-Ritz)
    const void* vf = nullptr;    // values in the filter precision
};

struct HBufs {
    double2 *Y, *Q, *T, *T2, *X, *Aq, *Bq, *Vr, *gpart;
    double *lam, *res, *rpart, *zw;
    int *mk, *status, *nactive, *perm;
    void* red;
    HArgs fa;  // filter arguments (vectors, lane state, partials)
    int nb;    // nodes per filter batch
    int ks;    // Gram split
    bool fp64;
    int* nactive_host;  // host copy of the two lane counters
    void* ozw;          // workspace of the sliced products (nullptr: FP64 DMMA products)
};

// One contour pass: Q = sum over all nodes (first pass: b = B Y, rii = 0) or
// the residual-inverse form (b = R, X, lam).  Returns 0 or -4; adds the BiCG
// steps launched to *iters and the lanes stopped by the iteration cap
// fpm(46) (inexact solves) to *capped.  The count of lanes still iterating is
// read back every kCheckSteps steps; lanes that stop in between idle.
constexpr int kCheckSteps = 8;

int h_filter_pass(HBufs& B, const HMat& A, const HMat& Bm, bool hasB, int m, int ne, int rii, const double2* b,
                  const double2* X, int maxit, double tol, long long* iters, long long* capped, cudaStream_t s)
{
    HArgs a = B.fa;
    a.n = A.n;
    a.m = m;
    a.ia = A.ia;
    a.ja = A.ja;
    a.av = A.vf;
    a.ib = hasB ? Bm.ia : nullptr;
    a.jb = hasB ? Bm.ja : nullptr;
    a.bv = hasB ? Bm.vf : nullptr;
    a.tol2 = tol * tol;
    for (int e0 = 0; e0 < ne; e0 += B.nb) {
        a.nb = std::min(B.nb, ne - e0);
        int nbp = 1;
        while (nbp < a.nb) nbp <<= 1;
        a.L = (long long)m * nbp;
        HCK(launch_h_init(a, B.fp64, b, X, B.zw + 4 * e0, B.lam, rii, ne, B.zw, e0 == 0 ? 1 : 0, s));
        HCK(cudaMemsetAsync(a.nactive + 1, 0, sizeof(int), s));
        int it = 0;
        while (it < maxit) {
            HCK(launch_h_step(a, B.fp64, maxit, s));
            ++it;
            if (it % kCheckSteps != 0 && it < maxit) continue;
            HCK(cudaMemcpyAsync(B.nactive_host, a.nactive, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            HCK(cudaStreamSynchronize(s));
            if (B.nactive_host[0] == 0) break;
        }
        *iters += it;
        *capped += B.nactive_host[1];
    }
    HCK(launch_h_fold(a, s));
    return 0;
}

}  // namespace

namespace {

// Device memory of one solve, carved from one workspace (256-byte aligned
// pieces): block vectors, reduced matrices, BiCG lane vectors and state, and
// the filter-precision copies of the values in mixed precision.
struct HPlan {
    int n = 0, m0 = 0, ne = 0, nb = 0, nbp = 0, ks = 1, nnz_a = 0, nnz_b = 0;
    long long Lmax = 0;
    bool fp64 = false, hasB = false;
    bool oz = true;  // fpm(54) = 0: projections and Ritz vectors from sliced BF16 products
};

HPlan h_plan(int n, int nnz_a, int nnz_b, int m0, const int* fpm)
{
    HPlan P;
    P.n = n;
    P.m0 = m0;
    P.ne = fpm[1];
    P.nnz_a = nnz_a;
    P.nnz_b = nnz_b;
    P.hasB = nnz_b > 0;
    P.fp64 = fpm[41] == 0;
    P.nb = std::min(P.ne, fpm[49] > 0 ? std::min(fpm[49], 32) : 16);
    P.nbp = 1;
    while (P.nbp < P.nb) P.nbp <<= 1;
    P.Lmax = (long long)m0 * P.nbp;
    h_gram_partial(n, m0, &P.ks);
    P.oz = fpm[53] == 0;
    return P;
}

struct HCarve {
    char* base;
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

// Carves B (and the filter-precision value copies af, bf) from base; with
// base == nullptr only measures.  Returns the bytes needed.
size_t h_carve(const HPlan& P, void* base, HBufs& B, float2** af, float2** bf)
{
    HCarve c{(char*)base};
    const size_t blk = (size_t)P.n * P.m0, mm = (size_t)P.m0 * P.m0;
    const size_t vb = P.fp64 ? sizeof(double2) : sizeof(float2);
    B.Y = c.take<double2>(blk);
    B.Q = c.take<double2>(blk);
    B.T = c.take<double2>(blk);
    B.X = c.take<double2>(blk);
    B.T2 = P.hasB ? c.take<double2>(blk) : nullptr;
    B.Aq = c.take<double2>(mm);
    B.Bq = c.take<double2>(mm);
    B.Vr = c.take<double2>(mm);
    B.gpart = c.take<double2>(h_gram_partial(P.n, P.m0, nullptr));
    B.lam = c.take<double>(P.m0);
    B.res = c.take<double>(P.m0);
    B.rpart = c.take<double>(h_resid_partial(P.n, P.m0));
    B.zw = c.take<double>(4 * (size_t)P.ne);
    B.mk = c.take<int>(1);
    B.status = c.take<int>(2);
    B.nactive = c.take<int>(2);
    B.perm = c.take<int>(P.m0);
    B.red = c.take<char>(h_reduced_work_bytes(P.m0));
    void** fv[6] = {&B.fa.r, &B.fa.rh, &B.fa.p, &B.fa.ph, &B.fa.q, &B.fa.qh};
    for (void** v : fv) *v = c.take<char>((size_t)P.n * P.Lmax * vb);
    B.fa.dQ = P.fp64 ? nullptr : c.take<float2>(blk);
    B.fa.st = c.take<HLane>(P.Lmax);
    B.fa.part = c.take<double2>((size_t)row_blocks(P.n) * 2 * P.Lmax);
    *af = P.fp64 ? nullptr : c.take<float2>(P.nnz_a);
    *bf = (P.fp64 || !P.hasB) ? nullptr : c.take<float2>(P.nnz_b);
    B.ozw = P.oz ? c.take<char>(h_sliced_work_bytes(P.n, P.m0)) : nullptr;
    return c.off + 256;
}

// The FEAST loop on device CSR data; x_dev: caller's column-major n x m0
// complex block (start subspace in, Ritz vectors out).  B: carved buffers.
int h_solve(const HMat& A, const HMat& Bm, bool hasB, int* fpm, double emin, double emax, int* m0io, double* e_host,
            double2* x_dev, int* M_out, double* res_host, double* epsout, int* loop_out, HBufs& B, cudaStream_t s)
{
    const int n = A.n, m0 = *m0io, ne = fpm[1];
    const double alpha = std::max(std::fabs(emin), std::fabs(emax));
    const double eps = std::pow(10.0, -fpm[2]);
    const double tol = std::pow(10.0, -fpm[44]);
    const int maxit = fpm[45], maxloop = fpm[3];
    std::vector<double> zw;
    contour_nodes(fpm[15], ne, emin, emax, fpm[17] / 100.0, zw);
    const size_t blk = (size_t)n * m0;
    B.fa.Q = B.Q;
    B.fa.nactive = B.nactive;
    int nact_host[2] = {0, 0};
    B.nactive_host = nact_host;
    HCK(cudaMemcpyAsync(B.zw, zw.data(), sizeof(double) * zw.size(), cudaMemcpyHostToDevice, s));
    HCK(cudaMemsetAsync(B.lam, 0, sizeof(double) * m0, s));
    long long iters = 0, capped = 0;
    int st = 0;
    if (fpm[4] == 1) {
        // a given subspace is tested by Rayleigh-Ritz before any filtering
        hk_col_to_row<<<grid_of((long long)blk), 256, 0, s>>>(n, m0, x_dev, B.Q);
        count_launches(1);
        HCK(cudaGetLastError());
    } else {
        const unsigned long long seed = fpm[51] ? (unsigned long long)fpm[51] : 0x5EEDull;
        hk_random<<<grid_of((long long)blk), 256, 0, s>>>((long long)blk, seed, B.Y);
        count_launches(1);
        HCK(cudaGetLastError());
        const double2* b = B.Y;
        if (hasB) {
            HCK(launch_h_spmm(n, m0, Bm.ia, Bm.ja, Bm.v, B.Y, B.T, s));
            b = B.T;
        }
        if ((st = h_filter_pass(B, A, Bm, hasB, m0, ne, 0, b, nullptr, maxit, tol, &iters, &capped, s))) return st;
    }
    std::vector<double> lam(m0), res(m0);
    int mk = m0, M = 0, info = 0, k = 0, stat[2] = {0, 0};
    double trace_prev = 0.0, eo = 1.0;
    char line[256];
    snprintf(line, sizeof(line), "#It |  #Eig  |          Trace            |     Error-Trace          |     Max-Residual\n");
    feast_log(fpm[0], line);
    for (k = 0;; ++k) {
        // Rayleigh-Ritz: Aq = Q^H A Q, Bq = Q^H B Q
        HCK(launch_h_spmm(n, m0, A.ia, A.ja, A.v, B.Q, B.T, s));
        auto gram = [&](const double2* Xg, const double2* Yg, double2* Cg) {
            return B.ozw ? launch_h_gram_sliced(n, m0, Xg, Yg, Cg, B.ozw, s)
                         : launch_h_gram(n, m0, Xg, Yg, Cg, B.gpart, B.ks, s);
        };
        HCK(gram(B.Q, B.T, B.Aq));
        if (hasB) {
            HCK(launch_h_spmm(n, m0, Bm.ia, Bm.ja, Bm.v, B.Q, B.T2, s));
            HCK(gram(B.Q, B.T2, B.Bq));
        } else {
            HCK(gram(B.Q, B.Q, B.Bq));
        }
        const int rst = h_reduced_gev(m0, B.Aq, B.Bq, B.lam, B.Vr, B.mk, B.status, B.red, s);
        if (rst == -4) return cuda_error(cudaGetLastError(), "reduced Hermitian eigensolver");
        if (rst) return cuda_error(cudaErrorInvalidValue, "reduced Hermitian eigensolver size");
        if (B.ozw) HCK(launch_h_gemm_sliced(n, m0, m0, B.Q, B.Vr, B.X, B.ozw, s));
        else HCK(launch_h_gemm(n, m0, m0, B.Q, B.Vr, B.X, s));
        HCK(launch_h_residual(n, m0, A.ia, A.ja, A.v, hasB ? Bm.ia : nullptr, hasB ? Bm.ja : nullptr,
                              hasB ? Bm.v : nullptr, B.X, B.lam, B.Y, B.rpart, B.res, alpha, s));
        HCK(cudaMemcpyAsync(lam.data(), B.lam, sizeof(double) * m0, cudaMemcpyDeviceToHost, s));
        HCK(cudaMemcpyAsync(res.data(), B.res, sizeof(double) * m0, cudaMemcpyDeviceToHost, s));
        HCK(cudaMemcpyAsync(&mk, B.mk, sizeof(int), cudaMemcpyDeviceToHost, s));
        HCK(cudaMemcpyAsync(stat, B.status, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
        HCK(cudaStreamSynchronize(s));
        if (mk < 1 || stat[0] != 0 || stat[1] != 0) { info = -3; break; }
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
        feast_log(fpm[0], line);
        if (capped) {
            snprintf(line, sizeof(line), "    %lld BiCG lanes stopped at the iteration cap fpm(46) = %d\n", capped,
                     maxit);
            feast_log(fpm[0], line);
            capped = 0;
        }
        const bool conv = M >= 1 && (fpm[5] == 1 ? maxres < eps : (k >= 1 && eo < eps));
        if (conv) { info = 0; break; }
        if (M == 0 && k >= 1) { info = 1; break; }
        if (k >= maxloop) { info = 2; break; }
        // residual-inverse pass on (X, Lambda), R = A X - B X Lambda in Y
        if ((st = h_filter_pass(B, A, Bm, hasB, m0, ne, 1, B.Y, B.X, maxit, tol, &iters, &capped, s))) return st;
    }
    fpm[59] = (int)std::min<long long>(iters, 2147483647LL);
    if (info == 0 && M >= mk) info = 3;
    if (info != -3) {
        std::vector<int> perm;
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
        HCK(cudaMemcpyAsync(B.perm, perm.data(), sizeof(int) * m0, cudaMemcpyHostToDevice, s));
        hk_gather_cols<<<grid_of((long long)blk), 256, 0, s>>>(n, m0, mk, B.X, B.perm, x_dev);
        count_launches(1);
        HCK(cudaGetLastError());
        HCK(cudaStreamSynchronize(s));
        *m0io = mk;
    }
    *M_out = M;
    *loop_out = k;
    *epsout = eo;
    return info;
}

}  // namespace

// ---------------------------------------------------------------- entry points
extern "C" size_t feast_hcsr_workspace_bytes(int n, int nnz_a, int nnz_b, int m0, const int* fpm)
{
    if (n <= 0 || m0 <= 0 || !fpm) return 0;
    HBufs B{};
    float2 *af = nullptr, *bf = nullptr;
    return h_carve(h_plan(n, nnz_a, nnz_b, m0, fpm), nullptr, B, &af, &bf);
}

static int h_dev_entry(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                       const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double emin, double emax,
                       int* m0, double* e, double* d_x, int* m, double* res, double* epsout, int* loop, int* info,
                       void* work, size_t work_bytes, cudaStream_t s)
{
    auto ret = [&](int v) { if (info) *info = v; return v; };
    if (n <= 0) return ret(202);
    if (!fpm) return ret(-109);
    int inf = fpm_check(fpm);
    if (inf) return ret(inf);
    if (fpm[13] != 0) return ret(114);  // one-pass modes: real symmetric driver only
    if (fpm[39] != 0) return ret(140);  // extreme-eigenvalue search: real symmetric driver only
    if (fpm[49] > 32) return ret(150);
    if (!(emin < emax)) return ret(200);
    if (!m0 || *m0 <= 0 || *m0 > n || *m0 > 1024) return ret(201);
    if (nnz_a < 0 || !d_ia || !d_ja || (nnz_a > 0 && !d_a)) return ret(-103);
    const bool hasB = d_ib != nullptr;
    if (hasB && (nnz_b < 0 || !d_jb || (nnz_b > 0 && !d_b))) return ret(-106);
    if (!e) return ret(-113);
    if (!d_x) return ret(-114);
    if (!m) return ret(-115);
    if (!res) return ret(-116);
    if (!epsout) return ret(-117);
    if (!loop) return ret(-118);
    const HPlan P = h_plan(n, nnz_a, hasB ? std::max(nnz_b, 1) : 0, *m0, fpm);
    HBufs B{};
    float2 *af = nullptr, *bf = nullptr;
    const size_t need = h_carve(P, nullptr, B, &af, &bf);
    if (work && work_bytes < need) return ret(-120);
    clear_last_error();
    HDevMem dm;
    if (!work) {  // no caller workspace: the library allocates it for this call
        char* w = nullptr;
        const cudaError_t ce = dm.alloc(&w, need);
        if (ce != cudaSuccess) return ret(cuda_error(ce, "workspace"));
        work = w;
    }
    h_carve(P, work, B, &af, &bf);
    B.fp64 = P.fp64;
    B.nb = P.nb;
    B.ks = P.ks;
    HMat A, Bm;
    A.n = n;
    A.nnz = nnz_a;
    A.ia = d_ia;
    A.ja = d_ja;
    A.v = (const double2*)d_a;
    A.vf = d_a;
    if (hasB) {
        Bm.n = n;
        Bm.nnz = nnz_b;
        Bm.ia = d_ib;
        Bm.ja = d_jb;
        Bm.v = (const double2*)d_b;
        Bm.vf = d_b;
    }
    if (!P.fp64) {  // complex float copies of the values for the filter
        cudaError_t ce = launch_h_cast(A.v, af, nnz_a, false, s);
        if (ce != cudaSuccess) return ret(cuda_error(ce, "cast"));
        A.vf = af;
        if (hasB) {
            if ((ce = launch_h_cast(Bm.v, bf, nnz_b, false, s)) != cudaSuccess) return ret(cuda_error(ce, "cast"));
            Bm.vf = bf;
        }
    }
    return ret(h_solve(A, Bm, hasB, fpm, emin, emax, m0, e, (double2*)d_x, m, res, epsout, loop, B, s));
}

extern "C" int feast_hcsr_solve_dev(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                                    const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double emin,
                                    double emax, int* m0, double* e, double* d_x, int* m, double* res,
                                    double* epsout, int* loop, int* info, void* d_work, size_t work_bytes,
                                    void* stream)
{
    return h_dev_entry(n, nnz_a, d_ia, d_ja, d_a, nnz_b, d_ib, d_jb, d_b, fpm, emin, emax, m0, e, d_x, m, res, epsout,
                       loop, info, d_work, work_bytes, (cudaStream_t)stream);
}

// Validates a host complex CSR (base ia[0] = 0 or 1; values interleaved
// (re, im)) and expands 'L' / 'U' storage to full rows: the mirrored entry of
// a_ij is conj(a_ij).  Rows are sorted by column.  arg0: position of the
// values argument, for the -(100 + i) codes.
static int host_hcsr(char uplo, int n, const double* v, const int* ia, const int* ja, int arg0, std::vector<int>& oia,
                     std::vector<int>& oja, std::vector<double2>& ov)
{
    if (!v) return -(100 + arg0);
    if (!ia) return -(100 + arg0 + 1);
    if (!ja) return -(100 + arg0 + 2);
    const int base = ia[0];
    if (base != 0 && base != 1) return -(100 + arg0 + 1);
    for (int i = 0; i < n; ++i)
        if (ia[i + 1] < ia[i]) return -(100 + arg0 + 1);
    std::vector<std::vector<std::pair<int, double2>>> rows(n);
    for (int i = 0; i < n; ++i)
        for (int p = ia[i] - base; p < ia[i + 1] - base; ++p) {
            const int j = ja[p] - base;
            if (j < 0 || j >= n) return -(100 + arg0 + 2);
            const double2 a = make_double2(v[2 * (size_t)p], v[2 * (size_t)p + 1]);
            if (!std::isfinite(a.x) || !std::isfinite(a.y)) return -(100 + arg0);
            if (uplo == 'L' && j > i) return -(100 + arg0 + 2);
            if (uplo == 'U' && j < i) return -(100 + arg0 + 2);
            rows[i].push_back({j, a});
            if (uplo != 'F' && j != i) rows[j].push_back({i, make_double2(a.x, -a.y)});
        }
    oia.assign(n + 1, 0);
    oja.clear();
    ov.clear();
    for (int i = 0; i < n; ++i) {
        std::stable_sort(rows[i].begin(), rows[i].end(),
                         [](const std::pair<int, double2>& x, const std::pair<int, double2>& y) { return x.first < y.first; });
        for (auto& pr : rows[i]) {
            oja.push_back(pr.first);
            ov.push_back(pr.second);
        }
        oia[i + 1] = (int)oja.size();
    }
    // The conjugate-shift shadow system assumes K^H = conj(z) B - A, i.e. a
    // Hermitian matrix: a real diagonal and, in full storage, a_ji = conj(a_ij)
    // (relative tolerance 1e-12, duplicate entries summed).  A mirrored
    // triangle is Hermitian off the diagonal by construction.
    auto entry = [&](int i, int j) {  // summed value of (i, j); zero if absent
        const auto first = std::lower_bound(oja.begin() + oia[i], oja.begin() + oia[i + 1], j);
        double2 sum = make_double2(0.0, 0.0);
        for (auto it = first; it != oja.begin() + oia[i + 1] && *it == j; ++it) {
            sum.x += ov[it - oja.begin()].x;
            sum.y += ov[it - oja.begin()].y;
        }
        return sum;
    };
    for (int i = 0; i < n; ++i) {
        const double2 d = entry(i, i);
        if (std::fabs(d.y) > 16.0 * 2.220446049250313e-16 * std::fabs(d.x)) return -(100 + arg0);
        if (uplo != 'F') continue;
        for (int p = oia[i]; p < oia[i + 1]; ++p) {
            const int j = oja[p];
            if (j == i) continue;
            const double2 a = entry(i, j), b = entry(j, i);
            const double diff = std::hypot(a.x - b.x, a.y + b.y);
            if (diff > 1e-12 * (std::hypot(a.x, a.y) + std::hypot(b.x, b.y))) return -(100 + arg0);
        }
    }
    return 0;
}

extern "C" int feast_hcsr_solve(char uplo, int n, const double* a, const int* ia, const int* ja, const double* b,
                                const int* ib, const int* jb, int* fpm, double emin, double emax, int* m0, double* e,
                                double* x, int* m, double* res, double* epsout, int* loop, int* info)
{
    auto ret = [&](int v) { if (info) *info = v; return v; };
    if (uplo != 'F' && uplo != 'L' && uplo != 'U') return ret(-101);
    if (n <= 0) return ret(202);
    if (!fpm) return ret(-109);
    int inf = fpm_check(fpm);
    if (inf) return ret(inf);
    if (fpm[13] != 0) return ret(114);
    if (fpm[39] != 0) return ret(140);
    if (fpm[49] > 32) return ret(150);
    if (!(emin < emax)) return ret(200);
    if (!m0 || *m0 <= 0 || *m0 > n || *m0 > 1024) return ret(201);
    if (!e) return ret(-113);
    if (!x) return ret(-114);
    if (!m) return ret(-115);
    if (!res) return ret(-116);
    if (!epsout) return ret(-117);
    if (!loop) return ret(-118);
    std::vector<int> aia, aja, bia, bja;
    std::vector<double2> av, bv;
    if ((inf = host_hcsr(uplo, n, a, ia, ja, 3, aia, aja, av))) return ret(inf);
    const bool hasB = b || ib || jb;
    if (hasB && (inf = host_hcsr(uplo, n, b, ib, jb, 6, bia, bja, bv))) return ret(inf);
    clear_last_error();
    const int mm0 = *m0;
    HDevMem dm;
    int *d_ia = nullptr, *d_ja = nullptr, *d_ib = nullptr, *d_jb = nullptr;
    double2 *d_a = nullptr, *d_b = nullptr, *d_x = nullptr;
#define HK2(x)                                                       \
    do {                                                             \
        cudaError_t _e = (x);                                        \
        if (_e != cudaSuccess) return ret(cuda_error(_e, #x));       \
    } while (0)
    HK2(dm.alloc(&d_ia, aia.size()));
    HK2(dm.alloc(&d_ja, aja.size()));
    HK2(dm.alloc(&d_a, av.size()));
    HK2(dm.alloc(&d_x, (size_t)n * mm0));
    HK2(cudaMemcpy(d_ia, aia.data(), sizeof(int) * aia.size(), cudaMemcpyHostToDevice));
    HK2(cudaMemcpy(d_ja, aja.data(), sizeof(int) * aja.size(), cudaMemcpyHostToDevice));
    HK2(cudaMemcpy(d_a, av.data(), sizeof(double2) * av.size(), cudaMemcpyHostToDevice));
    if (hasB) {
        HK2(dm.alloc(&d_ib, bia.size()));
        HK2(dm.alloc(&d_jb, bja.size()));
        HK2(dm.alloc(&d_b, bv.size()));
        HK2(cudaMemcpy(d_ib, bia.data(), sizeof(int) * bia.size(), cudaMemcpyHostToDevice));
        HK2(cudaMemcpy(d_jb, bja.data(), sizeof(int) * bja.size(), cudaMemcpyHostToDevice));
        HK2(cudaMemcpy(d_b, bv.data(), sizeof(double2) * bv.size(), cudaMemcpyHostToDevice));
    }
    if (fpm[4] == 1) HK2(cudaMemcpy(d_x, x, sizeof(double2) * (size_t)n * mm0, cudaMemcpyHostToDevice));
    inf = h_dev_entry(n, (int)aja.size(), d_ia, d_ja, (const double*)d_a, hasB ? (int)bja.size() : 0, d_ib, d_jb,
                      (const double*)d_b, fpm, emin, emax, m0, e, (double*)d_x, m, res, epsout, loop, info, nullptr, 0,
                      nullptr);
    if (inf >= 0 || inf == -3)
        HK2(cudaMemcpy(x, d_x, sizeof(double2) * (size_t)n * mm0, cudaMemcpyDeviceToHost));
#undef HK2
    return ret(inf);
}
