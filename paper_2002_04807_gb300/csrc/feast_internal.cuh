// Internal declarations shared by the CUDA translation units of libfeast_gb300.
// Nothing here is part of the public C ABI (include/feast_gb300.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace feast {

// ---------------------------------------------------------------- complex helpers
template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <typename T> using c2_t = typename C2<T>::type;

template <typename V> __device__ __forceinline__ V cmk(decltype(V::x) r, decltype(V::x) i) { V v; v.x = r; v.y = i; return v; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) { return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// a + b*c
template <typename V> __device__ __forceinline__ V cfma(V b, V c, V a) {
    return cmk<V>(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}

// ---------------------------------------------------------------- filter problem table
// One entry per independent eigenproblem handled by a filter launch.  All
// pointers are device pointers; row pointers are 0-based and local to the problem.
struct FiltProb {
    int n;              // rows
    int m0;             // subspace columns of this problem
    int G;              // column groups = ceil(m0 / Mt)
    int nrb;            // row blocks per group = ceil(n / RB)
    long long item0;    // first work item (items of one problem are contiguous: g-major, rb fastest)
    int nrb_b;          // row blocks per group of the streaming step = ceil(n / RBb)
    long long item0_b;  // first work item of the streaming step
    long long vec_off;  // offset of this problem's block vectors, in complex elements (G*n*W)
    int col_off;        // offset of this problem's columns in the per-column arrays (G*W)
    int grp_off;        // offset of this problem's groups in the per-group arrays (G)
    long long q_off;    // offset of this problem's FP64 n x m0 blocks (row-major)
    long long dq_off;   // offset of this problem's quadrature accumulator tiles ([G][n][mt])
    const int* ia;      // A row pointers [n+1]
    const int* ja;      // A column indices
    const void* av;     // A values (float or double, the filter's real type)
    const int* ib;      // B row pointers, or nullptr for B = I
    const int* jb;
    const void* bv;
    const int* app;     // A row pointers into apk, rows padded to chunks of 8 entries
    const void* apk;    // A as packed (column, value) entries: int2 (float) or int4 (double)
    const int* bpp;     // B padded row pointers (general B), or nullptr
    const void* bpk;    // B packed entries (general B), or nullptr
    const void* bd;     // B diagonal values in the filter's real type (diagonal B), or nullptr
    const double* zw;   // Ne nodes and weights, [Ne][4] = (Re z, Im z, Re w, Im w)
    const double* lam;  // Ritz values of the previous Rayleigh-Ritz step [m0]
    const int* mk;      // live subspace columns (device), or nullptr for m0
    int ne;             // number of contour nodes
    int active;         // 0: problem finished, its items are skipped
};

// Per-column COCG state (FP64 for stability of the scalar recurrences).
struct ColState {
    double2 rho;    // r^T r (unconjugated)
    double2 alpha;  // step length of the current iteration
    double2 beta;   // p update coefficient of the current iteration
    double2 z;      // shift z_e of the column's node
    double2 c;      // filter coefficient applied to the column's solution
    double2 ca;     // c * alpha
    double bn2;     // ||b||^2
    double rn2;     // ||r||^2 of the last iteration
    int active;     // 1 while the column iterates
    double rq;      // rho(lambda_m): filter value of the column's Ritz value
    int iters;      // iterations taken
    int status;     // 0 ok, 1 converged, 2 breakdown
};

// Partial sums of the COCG dot products: every work item writes its own slot
// of kPartStride x W doubles; buckets of kPartBucket consecutive items are
// summed by the CTA that completes the bucket, and the group total by the CTA
// that completes the last bucket, always in item order (deterministic).
constexpr int kPartBucket = 32;
__host__ __device__ inline int part_buckets(int nrb) { return (nrb + kPartBucket - 1) / kPartBucket; }
__host__ __device__ inline int part_slots(int nrb) { return nrb + part_buckets(nrb); }

struct FilterArgs {
    const FiltProb* probs;
    int nprob;
    long long nitems;
    int W;          // lanes (complex columns) per row of a group tile
    int nbp;        // node lanes per subspace column (power of two)
    int mt;         // subspace columns per group = W / nbp
    int RB;         // rows per work item of the gathering step
    int RBb;        // rows per work item of the streaming step
    long long nitems_b;  // work items of the streaming step
    int hasB;       // 1 when the problems have a B matrix (all or none)
    int bmode;      // 0: B = I, 1: B diagonal, 2: general B (same for all problems)
    int nslot;      // partial-sum slots per group, >= part_slots(nrb) and part_slots(nrb_b) of every problem
    int nbk;        // bucket counters per group, >= part_buckets(nrb) and part_buckets(nrb_b)
    void* r;        // residual block vectors (complex T)
    void* p0;       // search directions, ping
    void* p1;       // search directions, pong
    ColState* cs;   // per-column state
    double* part;   // partial sums, [group][nslot][4][W]: item slots, then bucket slots
    unsigned* bk_count;   // per-group, per-bucket finished-item counters [group][nbk], zero between launches
    unsigned* grp_count;  // per-group finished-bucket counters, zero between launches
    int* grp_done;  // per-group "no active column" flags
    double* Q;      // FP64 filter accumulator (row-major n x m0 per problem)
    void* dQ;       // per-pass accumulator of the quadrature sum, filter precision, [group][row][mt] tiles
    double tol2;    // squared relative COCG tolerance
    int* iter_max;  // per-problem max iteration reached
    int* groups_left;  // per-problem number of groups still iterating
    unsigned long long* work;  // group-iterations done (one per group per COCG step)
    const int* kdev;  // if set, the COCG step index is read from here (graph replay)
    const int* item_prob;    // several problems: problem of each gathering-step item (else nullptr)
    const int* item_prob_b;  // and of each streaming-step item
    // staged-window gather of step A (single problem; see win_build in k_filter.cu)
    const int4* whdr;   // per row block: (windows, staged rows, staged position of its first row, entries)
    const int2* wwin;   // per row block: kWinMax windows (first row, rows)
    const void* wpk;    // per row block, one region: local row pointers, then its packed entries with staged positions
    int wcapr;          // staged rows per CTA (largest over the row blocks)
    int wcape;          // staged entries per CTA (largest over the row blocks)
    int* werr;          // set to 1 when a CTA gave up waiting for its staged rows
    long long wlimit;   // that wait's limit in SM clock cycles
};

// Windows of one row block of the staged gather, at most kWinMax.
constexpr int kWinMax = 16;

// ---------------------------------------------------------------- launchers (k_filter.cu)
cudaError_t launch_cocg_step_a(const FilterArgs& a, bool fp64, int k, int grid, cudaStream_t s);
cudaError_t launch_cocg_step_b(const FilterArgs& a, bool fp64, int k, int grid, cudaStream_t s);
cudaError_t launch_filter_init(const FilterArgs& a, bool fp64, const double* R, const double* X, int rii,
                               int init_q, int grid, cudaStream_t s);
cudaError_t launch_colstate_init(const FilterArgs& a, int node0, int rii, cudaStream_t s);
cudaError_t launch_shifted_spmm(const FilterArgs& a, bool fp64, int grid, cudaStream_t s);
cudaError_t launch_cast_values(const double* src, float* dst, long long n, cudaStream_t s);
cudaError_t launch_advance(int* kdev, cudaStream_t s);
cudaError_t launch_fold_dq(const FilterArgs& a, long long max_total, bool fp64, cudaStream_t s);
cudaError_t launch_pack_csr(int n, const int* ia, const int* ja, const double* av, const int* pp, bool fp64, void* out,
                            cudaStream_t s);
cudaError_t launch_cast_diag(int n, const int* ia, const double* av, bool fp64, void* out, cudaStream_t s);
// Staged-window gather (k_filter.cu).  win_build: for every row block of rbw
// rows of the packed matrix (pp, pk), its windows (hdr, win) and, in one
// region of meta, its local row pointers and its entries rewritten with
// staged positions (bytes: rows of blocks x (rbw + 4) x 4 + the packed
// entries); stat[0] largest
// staged rows, stat[1] largest entry count of a row block, stat[2] row blocks
// that do not fit, stat[3] entries with a column outside [0, n) (stat zeroed
// by the caller).  win_smem_bytes: dynamic shared memory of step A for capr
// staged rows and cape entries; win_occupancy: resident CTAs per SM of that
// step A variant (0 when it does not exist or does not fit).
cudaError_t launch_win_build(int n, int rbw, const int* pp, const void* pk, bool fp64, void* meta, int4* hdr,
                             int2* win, int* stat, cudaStream_t s);
size_t win_smem_bytes(bool fp64, int W, int rbw, int capr, int cape);
int win_occupancy(bool fp64, int W, int bmode, int rbw, size_t smem);
cudaError_t launch_cocg_step_aw(const FilterArgs& a, bool fp64, int rbw, int k, int grid, size_t smem,
                                cudaStream_t s);
// Warp-specialized form of the staged step A (one CTA per SM: 16 consumer
// warps and a producer warp, two stages; complex FP32 with 32 lanes): dynamic
// shared memory, resident CTAs per SM (0: variant missing or too large), launch.
size_t ws_smem_bytes(int W, int rbw, int capr, int cape);
int ws_occupancy(bool fp64, int W, int bmode, int rbw, int groups, size_t smem);
cudaError_t launch_cocg_step_ws(const FilterArgs& a, int rbw, int k, int grid, size_t smem, cudaStream_t s);
// persistent grid size of the COCG kernels: SMs x resident CTAs per SM
int filter_grid(bool fp64, int W);
void filter_grids(bool fp64, int W, int* grid_a, int* grid_b);

// ---------------------------------------------------------------- Rayleigh-Ritz (k_rr.cu)
// Y = A X (and optionally Z = B X) for row-major n x m FP64 blocks.
cudaError_t launch_spmm_f64(int n, int m, const int* ia, const int* ja, const double* av,
                            const double* X, double* Y, cudaStream_t s);
// C (m x m) = X^T Y with X, Y row-major n x m; split-K partial buffer part
// [ksplit][m][m]; result symmetrised (C + C^T)/2 when sym != 0.
cudaError_t launch_gram_f64(int n, int m, const double* X, const double* Y, double* C,
                            double* part, int ksplit, int sym, cudaStream_t s);
size_t gram_partial_doubles(int n, int m, int* ksplit_out, int nsm);
// part [ksplit][m][m] (upper-triangle partials) -> C: summed in split order, mirrored
cudaError_t launch_gram_reduce(int m, const double* part, int ksplit, double* C, cudaStream_t s);
// C = X^T Y to FP64 accuracy from exact BF16 slice products (k_ozaki.cu); part:
// gram_oz_partial_doubles(n, m, ...) doubles, ex: gram_oz_work_bytes(m) bytes.
// full: every entry of X^T Y (no symmetry assumed) instead of the upper
// triangle mirrored.
size_t gram_oz_partial_doubles(int n, int m, int* ksplit_out, long long* rows_per_split, int nsm, bool full = false);
size_t gram_oz_work_bytes(int m);
cudaError_t launch_gram_oz(int n, int m, const double* X, const double* Y, double* C, double* part, int* ex,
                           cudaStream_t s, bool full = false);
// C (n x k) = A (n x m) V (m x k), row-major, FP64 accuracy from exact BF16
// slice products (k_ozaki.cu); work: gemm_oz_work_bytes(n, m, k) bytes.
size_t gemm_oz_work_bytes(int n, int m, int k);
cudaError_t launch_gemm_oz(int n, int m, int k, const double* A, const double* V, double* C, void* work,
                           cudaStream_t s);
// C (n x k) = A (n x m, row-major) * V (m x k, row-major)
cudaError_t launch_gemm_nn_f64(int n, int m, int k, const double* A, const double* V, double* C,
                               cudaStream_t s);
// R = AX - BX diag(lam) with per-column partial norms; res_j = ||R_j|| / (alpha ||BX_j||)
cudaError_t launch_residual_f64(int n, int m, const int* ia, const int* ja, const double* av,
                                const int* ib, const int* jb, const double* bv, const double* X,
                                const double* lam, double* R, double* part, unsigned* counter,
                                double* res, double alpha, cudaStream_t s);
size_t residual_partial_doubles(int n, int m);
// t[c] = sum_i X[i][c] Y[i][c] (row-major n x m), deterministic; part as for the residuals
cudaError_t launch_coldot_f64(int n, int m, const double* X, const double* Y, double* part, double* t,
                              cudaStream_t s);

// ---------------------------------------------------------------- reduced eigensolver (k_eig.cu)
// Symmetric eigen-decomposition of the m x m row-major matrix A (destroyed):
// eigenvalues ascending in lam, eigenvectors in the columns of V (row-major).
// Returns the number of sweeps (>= 0), or -1 when the sweep limit was hit,
// or -2 when a grid barrier timed out.  work: device scratch of
// jacobi_work_bytes(m).
size_t jacobi_work_bytes(int m);
int jacobi_eig_dev(int m, double* A, double* lam, double* V, void* work, cudaStream_t s,
                   int* sweeps_host);
// Reduced generalized problem; see k_eig.cu.  work: reduced_work_bytes(m).
size_t reduced_work_bytes(int m);
// spin limit (SM clock cycles) of the library's bounded grid barriers (feast_set_wait_limit)
long long wait_limit_cycles();
int reduced_gev_dev(int m, const double* Aq, const double* Bq, double* lam, double* V, int* mk,
                    void* work, cudaStream_t s);

// ---------------------------------------------------------------- gradient (k_grad.cu)
// grad[p] = sum_k w_k Xr[i_p][k] Xr[j_p][k], w_k = gw[k] (lam NULL) or -gw[k] lam[k];
// half != 0 doubles the off-diagonal entries (one stored triangle).
cudaError_t launch_eig_grad(int n, const int* ia, const int* ja, int m, const double* Xr,
                            const double* gw, double* grad, cudaStream_t s, const double* lam = nullptr,
                            int half = 0);

// ---------------------------------------------------------------- batched Rayleigh-Ritz (k_batch.cu)
// One entry per problem of a batch; all pointers device; offsets in doubles.
struct BProb {
    int n, m;             // rows, subspace columns
    long long row0;       // first row in the flattened row space of the batch
    long long q_off;      // offset of the problem's n x m FP64 blocks (row-major)
    long long c_off;      // offset of its m x m blocks
    long long gpart_off;  // offset of its Gram split-K partials (gram_ks x m x m)
    long long w_off;      // offset of its reduced-solver work (6 m*m + 4 m)
    int l_off;            // offset of its m-vectors (Ritz values, residuals)
    const int* ia;
    const int* ja;
    const double* av;
    const int* ib;        // B or nullptr for B = I
    const int* jb;
    const double* bv;
    int gram_b0, gram_ks, gram_T;  // Gram blocks: first block, row splits, 64-wide tiles per side
    int gemm_b0;          // first block of the Ritz-vector product
    int res_b0;           // first 256-row block of the residual kernel
    double alpha;         // residual normalisation max(|Emin|, |Emax|)
    int active;           // 0 once the problem has converged
};
cudaError_t launch_b_spmm(const BProb* pr, int np, long long rows, const double* X, double* Y, int useB, cudaStream_t s);
cudaError_t launch_b_gram(const BProb* pr, int np, int nblocks, int maxm, const double* X, const double* Y, double* part,
                          double* C, cudaStream_t s);
cudaError_t launch_b_gemm(const BProb* pr, int np, int nblocks, const double* A, const double* V, double* Out,
                          cudaStream_t s);
cudaError_t launch_b_residual(const BProb* pr, int np, int nblocks, const double* X, const double* lam, double* R,
                              double* part, double* res, cudaStream_t s);
cudaError_t launch_b_reduced(const BProb* pr, int np, const double* Aq, const double* Bq, double* lam, double* V,
                             int* mk, double* work, cudaStream_t s);

int num_sms();
// kernel launches issued by this library (all threads), for launch accounting
long long launch_count();
void count_launches(int k);

}  // namespace feast
