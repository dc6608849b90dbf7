// Internal declarations of the complex Hermitian path (k_herm.cu and
// herm_driver.cu).  Nothing here is part of the public C ABI.
#pragma once
#include <cuda_runtime.h>

namespace feast {
namespace herm {

// Per-lane BiCG state (lane = one (node, column) pair), FP64.
struct HLane {
    double2 rho;    // rh^H r of the current iteration
    double2 alpha;  // step length
    double2 beta;   // direction update coefficient (primal; the shadow uses its conjugate)
    double2 z;      // node z_e of the lane (the shadow system uses conj z_e)
    double2 c;      // filter coefficient of the primal solution (the shadow's is conj c)
    double bn2;     // |b|^2
    double rn2;     // |r|^2 of the last iteration
    double rhn2;    // |rh|^2 of the last iteration
    int active;     // 1 while the lane iterates
    int iters;      // iterations taken
    int status;     // 0 iterating, 1 converged, 2 breakdown, 3 inactive column, 4 iteration cap
};

struct HArgs {
    int n;          // rows
    int m;          // subspace columns of the pass (live columns)
    int nb;         // nodes of the batch (<= 32)
    long long L;    // lanes = m * nbp, nbp = nb rounded up to a power of two, node fastest
    const int* ia;  // A row pointers [n+1], 0-based
    const int* ja;  // A column indices
    const void* av; // A values, complex in the filter precision
    const int* ib;  // B row pointers, or nullptr for B = I
    const int* jb;
    const void* bv; // B values, complex in the filter precision
    void* r;        // residuals, n x L complex (row-major)
    void* rh;       // shadow residuals
    void* p;        // directions
    void* ph;       // shadow directions
    void* q;        // K p
    void* qh;       // K^H ph
    HLane* st;      // lane state [L]
    double2* part;  // partial sums [nrbk][2][L]
    double2* Q;     // FP64 quadrature block, n x m complex (row-major)
    void* dQ;       // complex FP32 accumulator of one contour pass, n x m (row-major), folded
                    // into Q after the pass (mixed precision); nullptr: steps add to Q
    double tol2;    // squared relative BiCG tolerance
    int* nactive;   // [0]: lanes still iterating after the last finish_b; [1]: lanes stopped by
                    // the iteration cap since the counter was last cleared (device)
};

constexpr int kRowsPerItem = 256;
__host__ __device__ inline int row_blocks(int n) { return (n + kRowsPerItem - 1) / kRowsPerItem; }

// ---------------------------------------------------------------- launchers (k_herm.cu)
// Setup of one node batch: lane state from the batch's nodes zwb [nb][4]
// (z re, z im, w re, w im) and, with rii, the Ritz values lam [m]
// (c = w / (z - lambda_j), else c = w); r = rh = b (n x m FP64) on every
// lane of a column; |b|^2 per lane.  With init_q the quadrature block Q
// starts at X rho(lam) (rii; rho over all ne_all nodes zw_all) or zero.
cudaError_t launch_h_init(const HArgs& a, bool fp64, const double2* b, const double2* X, const double* zwb,
                          const double* lam, int rii, int ne_all, const double* zw_all, int init_q, cudaStream_t s);
// One BiCG step (four launches); *a.nactive = lanes still iterating after it.
cudaError_t launch_h_step(const HArgs& a, bool fp64, int maxit, cudaStream_t s);
// Q += dQ (n x m complex) after a contour pass
cudaError_t launch_h_fold(const HArgs& a, cudaStream_t s);
// complex CSR values: double2 -> float2 (mixed precision) or copy
cudaError_t launch_h_cast(const double2* src, void* dst, long long n, bool fp64, cudaStream_t s);

// Rayleigh-Ritz, FP64 complex, row-major blocks
// Y = A X (n x m)
cudaError_t launch_h_spmm(int n, int m, const int* ia, const int* ja, const double2* av, const double2* X,
                          double2* Y, cudaStream_t s);
// C = X^H Y (m x m) with split-K partials part [ks][m][m]
size_t h_gram_partial(int n, int m, int* ks);
cudaError_t launch_h_gram(int n, int m, const double2* X, const double2* Y, double2* C, double2* part, int ks,
                          cudaStream_t s);
// C (n x k) = A (n x m) V (m x k)
cudaError_t launch_h_gemm(int n, int m, int k, const double2* A, const double2* V, double2* C, cudaStream_t s);
// The same two products from exact BF16 slice products on the real views of
// the complex blocks (k_ozaki.cu kernels); work: h_sliced_work_bytes(n, max(m, k)).
size_t h_sliced_work_bytes(int n, int m);
cudaError_t launch_h_gram_sliced(int n, int m, const double2* X, const double2* Y, double2* C, void* work,
                                 cudaStream_t s);
cudaError_t launch_h_gemm_sliced(int n, int m, int k, const double2* A, const double2* V, double2* C, void* work,
                                 cudaStream_t s);
// res_j = ||A x_j - lam_j B x_j|| / (alpha ||B x_j||); R = A x - lam B x
size_t h_resid_partial(int n, int m);
cudaError_t launch_h_residual(int n, int m, const int* ia, const int* ja, const double2* av, const int* ib,
                              const int* jb, const double2* bv, const double2* X, const double* lam, double2* R,
                              double* part, double* res, double alpha, cudaStream_t s);
// Reduced generalized Hermitian problem Aq v = lam Bq v (m x m row-major):
// eigenvalues ascending in lam [mk], V (m x m row-major, first mk columns),
// *mk_dev the kept size; status_dev[0] = -3 when B_Q has no positive
// eigenvalue (or -1: its Jacobi hit the sweep limit), status_dev[1] = -1 when
// the second Jacobi did.  Enqueues only; returns 0, -1 (m outside 1..1024) or
// -4 (launch error).  work: h_reduced_work_bytes(m).
size_t h_reduced_work_bytes(int m);
int h_reduced_gev(int m, const double2* Aq, const double2* Bq, double* lam, double2* V, int* mk_dev, int* status_dev,
                  void* work, cudaStream_t s);
// Hermitian eigen-decomposition of the leading k x k block of A (m x m
// row-major, destroyed; k = *kdev, or m when kdev is null; m <= 1024): lam
// ascending (zero beyond k), V (m x m) the unitary eigenvectors in the
// leading block and zero elsewhere, Vw m x m scratch.  status_dev: 0 ok,
// -1 sweep limit.
cudaError_t launch_h_jacobi(int m, double2* A, double2* Vw, double* lam, double2* V, const int* kdev, int* status_dev,
                            cudaStream_t s);

}  // namespace herm
}  // namespace feast
