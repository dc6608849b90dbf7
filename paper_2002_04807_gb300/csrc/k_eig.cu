// Reduced dense eigensolver of the Rayleigh-Ritz step (FEAST v4.0 guide,
// Sec. 1.1: the reduced problem is a small dense generalized symmetric
// eigenproblem A_Q v = lambda B_Q v, solved in FP64).
//
// Symmetric eigen-decomposition: two-sided cyclic Jacobi with the
// round-robin ("circle method") pair ordering, so each round rotates mp/2
// disjoint pairs at once.  Rotation of the pair (p,q) (Golub & Van Loan,
// symmetric Schur decomposition): tau = (a_qq - a_pp)/(2 a_pq),
// t = sign(tau)/(|tau| + sqrt(1+tau^2)), c = 1/sqrt(1+t^2), s = t c, and
// A <- J^T A J with J = [[c, s], [-s, c]] on columns (p, q).  Applying J_k^T
// on the left and J_l on the right of every 2x2 block (k,l) at once lets one
// thread update one block with no further synchronisation.
//
// GB300 has little FP64 throughput per SM, so the rounds are spread over many
// CTAs of one cooperative launch, with one grid barrier per round; the
// barrier spins on a global counter with a clock-based time limit and raises
// an error flag instead of hanging.
//
// Generalized problem, first route: D = diag(B_Q)^{-1/2}, D B_Q D = L L^T
// (one-CTA Cholesky), S = D L^{-T}, Jacobi on S^T A_Q S = W Lambda W^T,
// V = S W.  Taken when every pivot is positive and ||L^{-1}||_F^2 <= 1e8.
// Second route (B_Q singular or ill conditioned):
// D = diag(B_Q)^{-1/2}, Jacobi on D B_Q D = U diag(d) U^T,
// keep d_i > 1e-14 max d, S = D U_k diag(d_k)^{-1/2}, Jacobi on S^T A_Q S =
// W Lambda W^T, V = S W (V^T B_Q V = I).  Dropped directions stay in the
// m x m arrays as exact zero columns of S and get a sentinel eigenvalue, so
// they sort last and the live count mk is the number of non-sentinel values.
#include <atomic>

#include "chol.cuh"
#include "feast_internal.cuh"

namespace feast {

static constexpr double kSentinel = 1e300;
static constexpr int kMaxSweeps = 60;
static constexpr int kEigThreads = 256;

static constexpr int kMaxHalf = 4096;  // m <= 8192

struct GridBar {
    unsigned long long count;  // arrivals since launch; never reset
    int err;
    int pad;
};

struct JacWork {
    GridBar bar;
    double fro;
    int sweeps;
    int status;
};

// Spin limit of the grid barrier in SM clock cycles (about two seconds at
// 2 GHz); feast_set_wait_limit changes it for the launches that follow.
static constexpr long long kDefaultSpinCycles = 4000000000LL;
static std::atomic<long long> g_spin_cycles{kDefaultSpinCycles};
long long wait_limit_cycles() { return g_spin_cycles.load(); }

// Bounded grid barrier for a cooperative launch: each CTA adds one arrival to
// a counter that only grows, then waits until the counter reaches the end of
// its generation.  Returns false when any CTA spun longer than `limit` clock
// cycles or an earlier barrier failed (the error flag is then set for all).
__device__ __forceinline__ bool grid_sync(GridBar* b, long long limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = (*(volatile int*)&b->err == 0);
        if (good) {
            unsigned long long old;
            asm volatile("atom.add.release.gpu.u64 %0, [%1], 1;" : "=l"(old) : "l"(&b->count) : "memory");
            const unsigned long long target = (old / gridDim.x + 1) * gridDim.x;
            const long long t0 = clock64();
            for (;;) {
                unsigned long long cur;
                asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(cur) : "l"(&b->count) : "memory");
                if (cur >= target) break;
                if (*(volatile int*)&b->err) { good = 0; break; }
                if (clock64() - t0 > limit) {
                    atomicExch(&b->err, 1);
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

// round-robin partner table: slot 0 holds player 0, slot s >= 1 holds
// player 1 + ((s - 1 + r) mod (mp - 1)); pair k is (slot k, slot mp-1-k)
__device__ __forceinline__ int rr_player(int slot, int r, int mp)
{
    return slot == 0 ? 0 : 1 + (slot - 1 + r) % (mp - 1);
}

// One grid barrier per round: every CTA computes all mp/2 rotations of the
// round itself (identical inputs, identical code, so identical angles) into
// shared memory, then updates its share of the 2x2 blocks from the current
// copy of A into the other copy, so no CTA writes what another still reads.
// Rotation tables in dynamic shared memory: c, s, t (doubles), p, q (ints).
__global__ void __launch_bounds__(kEigThreads) jacobi_coop(int m, double* A, double* A2, double* V, double* lam,
                                                          double* Vout, JacWork* w, long long limit)
{
    extern __shared__ double rsh[];
    const int mp = m + (m & 1);
    const int half = mp / 2;
    double* rc = rsh;
    double* rs = rc + half;
    double* rt = rs + half;
    int* rp = (int*)(rt + half);
    int* rq = rp + half;
    __shared__ int any;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gsz = gridDim.x * blockDim.x;
    // V = I
    for (long long idx = gtid; idx < (long long)m * m; idx += gsz) V[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
    if (blockIdx.x == 0) {
        __shared__ double red[kEigThreads];
        double s = 0.0;
        for (long long idx = threadIdx.x; idx < (long long)m * m; idx += blockDim.x)
            s += fabs(A[idx]) < 1e299 ? A[idx] * A[idx] : 0.0;  // sentinels excluded
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) w->fro = sqrt(red[0]);
    }
    if (!grid_sync(&w->bar, limit)) return;
    const double absfloor = 1e-18 * *(volatile double*)&w->fro;
    double* cur = A;
    double* nxt = A2;
    int sweep = 0;
    for (; sweep < kMaxSweeps && mp >= 2; ++sweep) {
        if (threadIdx.x == 0) any = 0;
        __syncthreads();
        for (int r = 0; r < mp - 1; ++r) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int p = rr_player(k, r, mp), q = rr_player(mp - 1 - k, r, mp);
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, sn = 0.0, t = 0.0;
                if (q < m) {
                    const double apq = __ldcg(cur + (size_t)p * m + q);
                    const double app = __ldcg(cur + (size_t)p * m + p), aqq = __ldcg(cur + (size_t)q * m + q);
                    const double thr = fmax(1.1e-16 * sqrt(fabs(app * aqq)), absfloor);
                    if (fabs(apq) > thr) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                        any = 1;
                    }
                }
                rc[k] = c;
                rs[k] = sn;
                rt[k] = t;
                rp[k] = p;
                rq[k] = q;
            }
            __syncthreads();
            // 2x2 block (k, l): rows of pair k, columns of pair l, cur -> nxt
            for (long long idx = gtid; idx < (long long)half * half; idx += gsz) {
                const int k = (int)(idx / half), l = (int)(idx % half);
                const int p = rp[k], q = rq[k], pp = rp[l], qq = rq[l];
                const bool qv = q < m, qqv = qq < m;
                if (k == l) {  // diagonal block: closed form
                    const double app = __ldcg(cur + (size_t)p * m + p);
                    if (!qv) {
                        nxt[(size_t)p * m + p] = app;
                        continue;
                    }
                    const double apq = __ldcg(cur + (size_t)p * m + q), aqq = __ldcg(cur + (size_t)q * m + q);
                    if (rs[k] == 0.0) {
                        nxt[(size_t)p * m + p] = app;
                        nxt[(size_t)q * m + q] = aqq;
                        nxt[(size_t)p * m + q] = apq;
                        nxt[(size_t)q * m + p] = __ldcg(cur + (size_t)q * m + p);
                    } else {
                        nxt[(size_t)p * m + p] = app - rt[k] * apq;
                        nxt[(size_t)q * m + q] = aqq + rt[k] * apq;
                        nxt[(size_t)p * m + q] = 0.0;
                        nxt[(size_t)q * m + p] = 0.0;
                    }
                    continue;
                }
                const double ck = rc[k], sk = rs[k], cl = rc[l], sl = rs[l];
                const double x00 = __ldcg(cur + (size_t)p * m + pp);
                const double x01 = qqv ? __ldcg(cur + (size_t)p * m + qq) : 0.0;
                const double x10 = qv ? __ldcg(cur + (size_t)q * m + pp) : 0.0;
                const double x11 = (qv && qqv) ? __ldcg(cur + (size_t)q * m + qq) : 0.0;
                // rows: new row p = c row p - s row q ; new row q = s row p + c row q
                const double y00 = ck * x00 - sk * x10, y01 = ck * x01 - sk * x11;
                const double y10 = sk * x00 + ck * x10, y11 = sk * x01 + ck * x11;
                // columns: new col p' = c col p' - s col q' ; new col q' = s col p' + c col q'
                nxt[(size_t)p * m + pp] = cl * y00 - sl * y01;
                if (qqv) nxt[(size_t)p * m + qq] = sl * y00 + cl * y01;
                if (qv) nxt[(size_t)q * m + pp] = cl * y10 - sl * y11;
                if (qv && qqv) nxt[(size_t)q * m + qq] = sl * y10 + cl * y11;
            }
            for (long long idx = gtid; idx < (long long)m * half; idx += gsz) {
                const int i = (int)(idx / half), k = (int)(idx % half);
                const double sk = rs[k];
                if (sk == 0.0) continue;
                const double ck = rc[k];
                const int p = rp[k], q = rq[k];
                const double vp = V[(size_t)i * m + p], vq = V[(size_t)i * m + q];
                V[(size_t)i * m + p] = ck * vp - sk * vq;
                V[(size_t)i * m + q] = sk * vp + ck * vq;
            }
            if (!grid_sync(&w->bar, limit)) return;
            double* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        if (!any) break;  // same decision in every CTA
    }
    // ascending order: rank of each diagonal entry (ties by index)
    for (int i = gtid; i < m; i += gsz) {
        const double li = __ldcg(cur + (size_t)i * m + i);
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double lj = __ldcg(cur + (size_t)j * m + j);
            rank += (lj < li) || (lj == li && j < i);
        }
        lam[rank] = li;
        for (int row = 0; row < m; ++row) Vout[(size_t)row * m + rank] = V[(size_t)row * m + i];
    }
    if (gtid == 0) {
        w->sweeps = sweep;
        w->status = sweep >= kMaxSweeps ? -1 : 0;
    }
}

static size_t rot_smem(int m)
{
    const int half = (m + (m & 1)) / 2;
    return (size_t)half * (3 * sizeof(double) + 2 * sizeof(int));
}

size_t jacobi_work_bytes(int m)
{
    return 1024 + sizeof(JacWork) + 2 * sizeof(double) * (size_t)m * m;
}

static int coop_grid(int m)
{
    static const int per_sm = [] {  // initialised once, thread-safe
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, jacobi_coop, kEigThreads, rot_smem(2 * kMaxHalf));
        return v > 0 ? v : 1;
    }();
    const int mp = m + (m & 1);
    const long long work = (long long)m * (mp / 2) > (long long)(mp / 2) * (mp / 2) ? (long long)m * (mp / 2)
                                                                                    : (long long)(mp / 2) * (mp / 2);
    long long blocks = (work + kEigThreads - 1) / kEigThreads;
    const long long cap = (long long)num_sms() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks > num_sms()) blocks = num_sms();
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

static char* align256(char* p) { return (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255); }

// A (m x m, row-major) is destroyed; lam ascending; V row-major eigenvectors
// in columns.  m <= 8192 (the rotation tables of a round sit in shared
// memory); larger m returns -3.
int jacobi_eig_dev(int m, double* A, double* lam, double* V, void* work, cudaStream_t s, int* sweeps_host)
{
    if (m > 2 * kMaxHalf) return -3;
    char* p = align256((char*)work);
    JacWork* w = (JacWork*)p;
    p = align256(p + sizeof(JacWork));
    double* A2 = (double*)p;
    p = align256(p + sizeof(double) * (size_t)m * m);
    double* Vw = (double*)p;
    if (cudaMemsetAsync(w, 0, sizeof(JacWork), s) != cudaSuccess) return -3;
    const size_t smem = rot_smem(m);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(jacobi_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -3;
    int grid = coop_grid(m);
    long long limit = g_spin_cycles.load();
    void* args[] = {&m, &A, &A2, &Vw, &lam, &V, &w, &limit};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)jacobi_coop, dim3(grid), dim3(kEigThreads), args, smem, s);
    count_launches(1);
    if (e != cudaSuccess) return -3;
    if (sweeps_host) {
        JacWork h;
        if (cudaMemcpyAsync(&h, w, sizeof(JacWork), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -3;
        if (cudaStreamSynchronize(s) != cudaSuccess) return -3;
        *sweeps_host = h.sweeps;
        if (h.bar.err) return -2;
        if (h.status) return -1;
    }
    return 0;
}

// ---------------------------------------------------------------- generalized problem
__global__ void rg_scale(int m, const double* Aq, const double* Bq, double* At, double* Bt, double* dsc)
{
    const long long total = (long long)m * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / m), j = (int)(idx % m);
        const double bi = Bq[(size_t)i * m + i], bj = Bq[(size_t)j * m + j];
        const double di = bi > 0.0 ? 1.0 / sqrt(bi) : 0.0, dj = bj > 0.0 ? 1.0 / sqrt(bj) : 0.0;
        Bt[idx] = 0.5 * (Bq[(size_t)i * m + j] + Bq[(size_t)j * m + i]) * di * dj;
        At[idx] = 0.5 * (Aq[(size_t)i * m + j] + Aq[(size_t)j * m + i]);
        if (j == 0) dsc[i] = di;
    }
}

// S[r][c] = dsc[r] U[r][c] / sqrt(d_c) for kept c (d_c > 1e-14 max d), else 0.
__global__ void rg_basis(int m, const double* d, const double* U, const double* dsc, double* S, int* mk)
{
    const double dmax = d[m - 1];
    const long long total = (long long)m * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / m), c = (int)(idx % m);
        const bool keep = dmax > 0.0 && d[c] > 1e-14 * dmax;
        S[idx] = keep ? dsc[r] * U[idx] / sqrt(d[c]) : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int k = 0;
        for (int c = 0; c < m; ++c) k += (dmax > 0.0 && d[c] > 1e-14 * dmax);
        *mk = k;
    }
}

// Dropped directions (zero columns of S) get the sentinel on the diagonal.
__global__ void rg_sentinel(int m, const double* S, double* C)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        bool zero = true;
        for (int r = 0; r < m && zero; ++r) zero = S[(size_t)r * m + c] == 0.0;
        if (zero) C[(size_t)c * m + c] = kSentinel;
    }
}

// Cholesky route: factor B~ = L L^T in shared memory when (m^2 + 2m) doubles
// fit, else in the global scratch G; S = D X^T with X = L^{-1};
// status = 0 when accepted (and *mk = m), 1 otherwise.
static constexpr int kCholThreads = 1024;
static constexpr size_t kCholSmemMax = 224 * 1024;

__global__ void __launch_bounds__(kCholThreads) rg_cholinv(int m, const double* __restrict__ Bt,
                                                           const double* __restrict__ dsc, double* __restrict__ S,
                                                           double* G, int use_smem, int* status, int* mk)
{
    extern __shared__ double sh[];
    __shared__ double red[kCholThreads / 32];
    double* M = use_smem ? sh : G;
    double* xd = M + (size_t)m * m;
    double* cj = xd + m;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) M[idx] = Bt[idx];
    __syncthreads();
    const bool ok = cta_chol_inv(m, M, xd, cj, red);
    if (ok) {
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int r = idx / m, c = idx % m;
            S[idx] = c > r ? dsc[r] * M[idx] : (c == r ? dsc[r] * xd[r] : 0.0);
        }
    }
    if (threadIdx.x == 0) {
        *status = ok ? 0 : 1;
        if (ok) *mk = m;
    }
}

static size_t chol_bytes(int m) { return ((size_t)m * m + 2 * (size_t)m) * sizeof(double); }

size_t reduced_work_bytes(int m)
{
    const size_t mm = (size_t)m * m * sizeof(double);
    int ks = 0;
    const size_t gp = gram_partial_doubles(m, m, &ks, num_sms()) * sizeof(double);
    return 8 * (mm + 256) + (m * sizeof(double) + 256) * 2 + gp + 256 + jacobi_work_bytes(m) + chol_bytes(m) +
           512 + 1024;
}

// lam[m] (ascending, sentinels >= 1e299 last), V row-major m x m, *mk (device).
// Synchronises the stream to check the two Jacobi runs.  Returns 0, -3 when
// a Jacobi run did not converge or its grid barrier timed out, -4 on a CUDA
// error.
int reduced_gev_dev(int m, const double* Aq, const double* Bq, double* lam, double* V, int* mk, void* work,
                    cudaStream_t s)
{
    int sweeps = 0;
    const size_t mm = (size_t)m * m;
    char* p = align256((char*)work);
    auto take = [&](size_t bytes) { char* q = p; p = align256(p + bytes); return q; };
    double* At = (double*)take(mm * 8);
    double* Bt = (double*)take(mm * 8);
    double* U = (double*)take(mm * 8);
    double* S = (double*)take(mm * 8);
    double* T1 = (double*)take(mm * 8);
    double* C = (double*)take(mm * 8);
    double* W = (double*)take(mm * 8);
    double* d = (double*)take(m * 8);
    double* dsc = (double*)take(m * 8);
    int ks = 0;
    const size_t gp = gram_partial_doubles(m, m, &ks, num_sms());
    double* gpart = (double*)take(gp * 8);
    void* jw = take(jacobi_work_bytes(m));
    double* G = (double*)take(chol_bytes(m));
    int* cst = (int*)take(256);
    const int blocks = (int)((mm + 255) / 256 < 1024 ? (mm + 255) / 256 : 1024);
    rg_scale<<<blocks, 256, 0, s>>>(m, Aq, Bq, At, Bt, dsc);
    count_launches(2);  // scale, Cholesky
    if (cudaGetLastError() != cudaSuccess) return -4;
    const int use_smem = chol_bytes(m) <= kCholSmemMax;
    if (use_smem && cudaFuncSetAttribute(rg_cholinv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chol_bytes(m)) != cudaSuccess)
        return -4;
    rg_cholinv<<<1, kCholThreads, use_smem ? chol_bytes(m) : 0, s>>>(m, Bt, dsc, S, G, use_smem, cst, mk);
    if (cudaGetLastError() != cudaSuccess) return -4;
    int hst = 1;
    if (cudaMemcpyAsync(&hst, cst, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -4;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -4;
    if (hst == 0) {
        if (launch_gemm_nn_f64(m, m, m, At, S, T1, s) != cudaSuccess) return -4;
        if (launch_gram_f64(m, m, S, T1, C, gpart, ks, 1, s) != cudaSuccess) return -4;
        const int st = jacobi_eig_dev(m, C, lam, W, jw, s, &sweeps);
        if (st) return st == -3 ? -4 : -3;
        if (launch_gemm_nn_f64(m, m, m, S, W, V, s) != cudaSuccess) return -4;
        return 0;
    }
    count_launches(2);  // basis, sentinel
    int st = jacobi_eig_dev(m, Bt, d, U, jw, s, &sweeps);
    if (st) return st == -3 ? -4 : -3;
    rg_basis<<<blocks, 256, 0, s>>>(m, d, U, dsc, S, mk);
    if (cudaGetLastError() != cudaSuccess) return -4;
    if (launch_gemm_nn_f64(m, m, m, At, S, T1, s) != cudaSuccess) return -4;
    if (launch_gram_f64(m, m, S, T1, C, gpart, ks, 1, s) != cudaSuccess) return -4;
    rg_sentinel<<<(m + 255) / 256, 256, 0, s>>>(m, S, C);
    if (cudaGetLastError() != cudaSuccess) return -4;
    st = jacobi_eig_dev(m, C, lam, W, jw, s, &sweeps);
    if (st) return st == -3 ? -4 : -3;
    if (launch_gemm_nn_f64(m, m, m, S, W, V, s) != cudaSuccess) return -4;
    return 0;
}

}  // namespace feast

extern "C" long long feast_set_wait_limit(long long cycles)
{
    return feast::g_spin_cycles.exchange(cycles >= 1 ? cycles : feast::kDefaultSpinCycles);
}
