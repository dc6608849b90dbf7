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
// thread update one block with no further synchronisation, so a round is
// "angles, barrier, block updates, barrier".
//
// GB300 has little FP64 throughput per SM, so the rounds are spread over many
// CTAs of one cooperative launch; its grid barrier spins on a global counter
// with a clock-based time limit and raises an error flag instead of hanging.
//
// Generalized problem: D = diag(B_Q)^{-1/2}, Jacobi on D B_Q D = U diag(d) U^T,
// keep d_i > 1e-14 max d, S = D U_k diag(d_k)^{-1/2}, Jacobi on S^T A_Q S =
// W Lambda W^T, V = S W (V^T B_Q V = I).  Dropped directions stay in the
// m x m arrays as exact zero columns of S and get a sentinel eigenvalue, so
// they sort last and the live count mk is the number of non-sentinel values.
#include "feast_internal.cuh"

namespace feast {

static constexpr double kSentinel = 1e300;
static constexpr int kMaxSweeps = 60;
static constexpr int kEigThreads = 256;

struct GridBar {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

struct JacWork {
    GridBar bar;
    double fro;
    int sweeps;
    int status;
    int flags[kMaxSweeps];  // "a rotation happened in this sweep"
};

// Bounded grid barrier for a cooperative launch.  Returns false when any CTA
// timed out (about two seconds of spinning) or an earlier barrier failed.
__device__ __forceinline__ bool grid_sync(GridBar* b)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* genp = &b->gen;
        volatile int* errp = &b->err;
        int good = (*errp == 0);
        if (good) {
            const unsigned g = *genp;
            __threadfence();
            if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
                b->count = 0;
                __threadfence();
                atomicAdd(&b->gen, 1u);
            } else {
                const long long t0 = clock64();
                while (*genp == g) {
                    if (*errp) { good = 0; break; }
                    if (clock64() - t0 > 4000000000LL) {
                        atomicExch(&b->err, 1);
                        good = 0;
                        break;
                    }
                }
            }
            __threadfence();
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

// Rotation record of pair k: c, s, t, and the (p, q) players with p < q.
struct Rot {
    double c, s, t;
    int p, q;
};

__global__ void __launch_bounds__(kEigThreads) jacobi_coop(int m, double* A, double* V, double* lam,
                                                          double* Vout, JacWork* w, Rot* rot)
{
    const int mp = m + (m & 1);
    const int half = mp / 2;
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
    if (!grid_sync(&w->bar)) return;
    const double absfloor = 1e-18 * w->fro;
    int sweep = 0;
    for (; sweep < kMaxSweeps && mp >= 2; ++sweep) {
        for (int r = 0; r < mp - 1; ++r) {
            for (int k = gtid; k < half; k += gsz) {
                int p = rr_player(k, r, mp), q = rr_player(mp - 1 - k, r, mp);
                if (p > q) { const int t = p; p = q; q = t; }
                Rot R;
                R.p = p;
                R.q = q;
                R.c = 1.0;
                R.s = 0.0;
                R.t = 0.0;
                if (q < m) {
                    const double apq = A[(size_t)p * m + q];
                    const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                    const double thr = fmax(1.1e-16 * sqrt(fabs(app * aqq)), absfloor);
                    if (fabs(apq) > thr) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        R.c = 1.0 / sqrt(1.0 + t * t);
                        R.s = t * R.c;
                        R.t = t;
                        w->flags[sweep] = 1;
                    }
                }
                rot[k] = R;
            }
            if (!grid_sync(&w->bar)) return;
            // 2x2 block (k, l): rows of pair k, columns of pair l
            for (long long idx = gtid; idx < (long long)half * half; idx += gsz) {
                const int k = (int)(idx / half), l = (int)(idx % half);
                const Rot Rk = rot[k], Rl = rot[l];
                if (Rk.s == 0.0 && Rl.s == 0.0) continue;
                const int p = Rk.p, q = Rk.q, pp = Rl.p, qq = Rl.q;
                if (k == l) {  // diagonal block: closed form
                    if (Rk.s == 0.0) continue;
                    const double apq = A[(size_t)p * m + q];
                    A[(size_t)p * m + p] -= Rk.t * apq;
                    A[(size_t)q * m + q] += Rk.t * apq;
                    A[(size_t)p * m + q] = 0.0;
                    A[(size_t)q * m + p] = 0.0;
                    continue;
                }
                const bool qv = q < m, qqv = qq < m;
                const double x00 = A[(size_t)p * m + pp];
                const double x01 = qqv ? A[(size_t)p * m + qq] : 0.0;
                const double x10 = qv ? A[(size_t)q * m + pp] : 0.0;
                const double x11 = (qv && qqv) ? A[(size_t)q * m + qq] : 0.0;
                // rows: new row p = c row p - s row q ; new row q = s row p + c row q
                const double y00 = Rk.c * x00 - Rk.s * x10, y01 = Rk.c * x01 - Rk.s * x11;
                const double y10 = Rk.s * x00 + Rk.c * x10, y11 = Rk.s * x01 + Rk.c * x11;
                // columns: new col p' = c col p' - s col q' ; new col q' = s col p' + c col q'
                A[(size_t)p * m + pp] = Rl.c * y00 - Rl.s * y01;
                if (qqv) A[(size_t)p * m + qq] = Rl.s * y00 + Rl.c * y01;
                if (qv) A[(size_t)q * m + pp] = Rl.c * y10 - Rl.s * y11;
                if (qv && qqv) A[(size_t)q * m + qq] = Rl.s * y10 + Rl.c * y11;
            }
            for (long long idx = gtid; idx < (long long)m * half; idx += gsz) {
                const int i = (int)(idx / half), k = (int)(idx % half);
                const Rot Rk = rot[k];
                if (Rk.s == 0.0) continue;
                const double vp = V[(size_t)i * m + Rk.p], vq = V[(size_t)i * m + Rk.q];
                V[(size_t)i * m + Rk.p] = Rk.c * vp - Rk.s * vq;
                V[(size_t)i * m + Rk.q] = Rk.s * vp + Rk.c * vq;
            }
            if (!grid_sync(&w->bar)) return;
        }
        if (!((volatile int*)w->flags)[sweep]) break;
    }
    // ascending order: rank of each diagonal entry (ties by index)
    for (int i = gtid; i < m; i += gsz) {
        const double li = A[(size_t)i * m + i];
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double lj = A[(size_t)j * m + j];
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

size_t jacobi_work_bytes(int m)
{
    const int mp = m + (m & 1);
    return 1024 + sizeof(JacWork) + sizeof(Rot) * (size_t)(mp / 2 + 1) + sizeof(double) * (size_t)m * m;
}

static int coop_grid(int m)
{
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop, kEigThreads, 0);
        if (per_sm < 1) per_sm = 1;
    }
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

// A (m x m, row-major) is destroyed; lam ascending; V row-major eigenvectors in columns.
int jacobi_eig_dev(int m, double* A, double* lam, double* V, void* work, cudaStream_t s, int* sweeps_host)
{
    char* p = align256((char*)work);
    JacWork* w = (JacWork*)p;
    p = align256(p + sizeof(JacWork));
    Rot* rot = (Rot*)p;
    const int mp = m + (m & 1);
    p = align256(p + sizeof(Rot) * (size_t)(mp / 2 + 1));
    double* Vw = (double*)p;
    if (cudaMemsetAsync(w, 0, sizeof(JacWork), s) != cudaSuccess) return -3;
    int grid = coop_grid(m);
    void* args[] = {&m, &A, &Vw, &lam, &V, &w, &rot};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)jacobi_coop, dim3(grid), dim3(kEigThreads), args, 0, s);
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

size_t reduced_work_bytes(int m)
{
    const size_t mm = (size_t)m * m * sizeof(double);
    int ks = 0;
    const size_t gp = gram_partial_doubles(m, m, &ks, num_sms()) * sizeof(double);
    return 8 * (mm + 256) + (m * sizeof(double) + 256) * 2 + gp + 256 + jacobi_work_bytes(m) + 1024;
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
    const int blocks = (int)((mm + 255) / 256 < 1024 ? (mm + 255) / 256 : 1024);
    rg_scale<<<blocks, 256, 0, s>>>(m, Aq, Bq, At, Bt, dsc);
    count_launches(3);  // scale, basis, sentinel
    if (cudaGetLastError() != cudaSuccess) return -4;
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
