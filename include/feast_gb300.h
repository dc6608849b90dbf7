/*
 * feast_gb300.h -- C ABI of the GB300 (sm_103a) FEAST contour-filter eigensolver
 * for real symmetric sparse problems  A x = lambda B x  (B symmetric positive
 * definite; B = I when no B is given).
 *
 * Method: FEAST v4.0 user guide (Polizzi et al.), Sec. 1.1 "The FEAST
 * Algorithm": a subspace iteration that filters a block of M0 vectors with the
 * quadrature of the spectral projector along a half contour around
 * [Emin, Emax] (one shifted solve (z_e B - A) Y_e = RHS per node z_e), then
 * does a Rayleigh-Ritz step on the filtered block.  Sec. 3.1 (tips) describes
 * the residual inverse iteration that lets the shifted solves run in single
 * precision; Sec. 3.2 gives the driver arguments; Sec. 3.5 (IFEAST) the
 * iterative inner solver.  Sec. 4.1 describes the CSR storage.
 *
 * Conventions shared by every entry point:
 *  - fpm is the 64-entry parameter array of the guide's parameter table
 *    (Sec. 3.1), C indexing fpm[i-1] = fpm(i).  Used entries:
 *      fpm(1)  0 silent, 1 per-iteration log on stdout, n<0 append to feast<|n|>.log
 *      fpm(2)  Ne, number of half-contour nodes (Gauss and Zolotarev: 1..20, 24,
 *              32, 40, 48, 56; trapezoidal: 1..1024)
 *      fpm(3)  stopping tolerance 10^-fpm(3) on the relative residual (0..16)
 *      fpm(4)  maximum number of refinement loops (>= 0)
 *      fpm(5)  1: X holds the start subspace on entry; 0: a random start block
 *      fpm(6)  must be 1 (relative residual criterion)
 *      fpm(14) 0 normal run; 1 return the block Q after one contour pass
 *              (info 4); 2 stochastic estimate of the number of eigenvalues
 *              inside the contour (info 5), see feast_scsr_solve
 *      fpm(16) 0 Gauss-Legendre nodes, 1 trapezoidal nodes, 2 Zolotarev nodes
 *              (see feast_contour_nodes_rule)
 *      fpm(18) ellipse ratio in percent (> 0)
 *      fpm(40) 0 search interval given (feast_scsr_solve*); -1 / +1 search
 *              the M0/2 lowest / largest eigenpairs (feast_scsr_extreme*)
 *      fpm(42) 1: complex FP32 shifted solves (mixed precision), 0: complex FP64
 *      fpm(45) inner solver tolerance 10^-fpm(45) (0..16)
 *      fpm(46) inner solver iteration cap (>= 1)
 *      fpm(60) output: total number of inner (COCG) iterations
 *    Library options in reserved slots (0 = automatic):
 *      fpm(50) contour nodes solved at once (node batch); fpm(51) rows per
 *      inner-solver work item (0: the single-problem drivers stage the rows
 *      each item gathers in shared memory, 32 to 64 rows per item, when the
 *      matrix's row blocks read few contiguous column ranges and B is the
 *      identity or diagonal; else 256; > 0: that many rows, gathered through
 *      the caches); fpm(52) seed of the random start block;
 *      fpm(53) 1 = record per-kernel timings (see feast_last_profile);
 *      fpm(54) arithmetic of the Rayleigh-Ritz projections and Ritz vectors
 *      of the single-problem real and Hermitian drivers: 0 (default) =
 *      FP64-accurate sums of exact BF16 slice products on the tensor cores
 *      (feast_gram_oz_dev, feast_gemm_oz_dev; complex blocks through their
 *      real views), 1 = FP64 tensor cores (mma.sync m8n8k4 f64).  The
 *      batched driver uses the FP64 tensor cores.
 *  - Return value = info (also stored in *info where that argument exists),
 *    codes of the guide's info table (Sec. 3.1): 0 success; warnings 1 (no
 *    eigenvalue in the interval), 2 (no convergence within fpm(4) loops),
 *    3 (M0 too small: all Ritz values inside), 4 (only the filtered
 *    subspace returned, fpm(14)=1), 5 (only the stochastic eigenvalue count
 *    returned, fpm(14)=2), 7 (the search for extreme eigenvalues failed; the
 *    interval must be given); errors 200 (Emin >= Emax),
 *    201 (bad M0), 202 (bad N), 100+i (bad fpm(i)), -(100+i) (bad i-th
 *    argument, e.g. CSR indices out of range, non-finite values), -2 (inner
 *    solver failure), -3 (reduced eigensolver failure, e.g. B not positive
 *    definite).  Library extension: -4 = CUDA runtime error (message in
 *    feast_last_error()).
 *  - "Host" arguments are ordinary CPU memory owned by the caller; "device"
 *    arguments are CUDA global memory of the current device owned by the
 *    caller; stream is a cudaStream_t passed as void* (NULL = legacy stream).
 *    Entry points taking a stream enqueue work on it and return after the
 *    results they report on the host are available.
 *  - Dense blocks of vectors are column-major N x M0 (X(i,j) at x[i + N*j]) in
 *    the host/driver entry points, as in the guide; the kernel-level entry
 *    points state their own layouts.
 */
#ifndef FEAST_GB300_H
#define FEAST_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Fill fpm[0..63] with the defaults of the guide's parameter table (Sec. 3.1,
 * "feastinit").  Returns 0. */
int feast_init(int* fpm);

/* Text of the last CUDA error seen by this library in the calling thread
 * (empty when none).  The pointer stays valid until the next call. */
const char* feast_last_error(void);

/* Half-contour Gauss-Legendre nodes and weights (guide Sec. 4.2 "Search
 * contour", fpm(16)=0): z_e = c + r cos(t_e) + i a r sin(t_e),
 * w_e = (omega_e r / 2)(a cos(t_e) + i sin(t_e)), t_e = (pi/2)(1 - x_e),
 * c = (Emin+Emax)/2, r = (Emax-Emin)/2, a = ratio_pct/100, (x_e, omega_e)
 * the Gauss-Legendre rule on [-1,1] with x descending.  z and w are host
 * arrays of 2*ne doubles, (re, im) interleaved.  Returns 0, 102 for a bad ne,
 * 200 for emin >= emax. */
int feast_contour_nodes(int ne, double emin, double emax, int ratio_pct, double* z, double* w);

/* Nodes and weights of the quadrature rule fpm(16) = rule (guide Sec. 3.1,
 * parameter table: 0 Gauss-Legendre, 1 trapezoidal, 2 Zolotarev).  Gauss and
 * trapezoidal lie on the half ellipse of ratio_pct: a rule with nodes t_e in
 * [0, pi] and t-weights v_e gives w_e = (v_e r / pi)(a cos(t_e) + i sin(t_e));
 * the trapezoidal rule takes the midpoints t_e = pi (e - 1/2) / ne,
 * v_e = pi / ne (with the conjugate half, 2 ne equally spaced points of the
 * whole contour; on a circle its filter is 1 / (1 + ((lambda - c)/r)^(2 ne))).
 * Zolotarev (the guide cites Guettel, Polizzi, Tang and Viaud; ratio_pct not
 * used): with x = (lambda - c)/r, the filter is the best uniform rational
 * approximation of the interval's indicator outside the edge bands
 * 1/(1.05) < |x| < 1.05, built from Zolotarev's best approximation of the
 * sign function through u = (1 + x)/(1 - x); its ne conjugate pole pairs lie
 * on the circle through Emin and Emax and its error equioscillates (constant
 * term rho(inf), below half that error, left out).  rule 0 equals
 * feast_contour_nodes.  Returns 0, 116 for another rule, 102 for a bad ne
 * (trapezoidal: 1..1024; otherwise the Gauss counts), 200 for emin >= emax. */
int feast_contour_nodes_rule(int rule, int ne, double emin, double emax, int ratio_pct, double* z, double* w);

/* Timings of the last solve entry point (feast_scsr_solve*, feast_scsr_extreme*)
 * of the calling thread run with fpm(53) = 1 (all zero otherwise; an
 * extreme-eigenvalue search reports the totals of its solves), measured with CUDA events
 * on the solve's stream.  out (host, 20 doubles): [0] ms in COCG step A
 * launches, [1] ms in COCG step B launches, [2] step A launches, [3] step B
 * launches, [4] group-iterations (column groups x COCG steps done), [5] ms in
 * filter passes, [6] ms projecting (A Q, Q^T A Q, Q^T B Q), [7] ms in the
 * reduced eigensolver, [8] ms forming Ritz vectors and residuals, [9] tile
 * width W, [10] columns per group mt, [11] n, [12] bytes per complex value,
 * [13] column groups, [14] refinement loops, [15] kernel launches issued,
 * [16] rows per step-A work item, [17] 0 when step A gathers through the
 * caches, 1 when it stages the rows it gathers in shared memory (windows of r
 * copied by the bulk-copy engine), 2 for the staged form with a producer warp
 * and two stages (one CTA per SM), [18] step A CTAs (staged forms), [19]
 * staged rows per row block (staged forms).
 * Library extension (the guide reports phase timings only as a text log).
 * Returns 0. */
int feast_last_profile(double* out);

/* ---------------------------------------------------------------- drivers */

/* FEAST for a real symmetric CSR problem (guide Sec. 3.2, dfeast_scsrev /
 * dfeast_scsrgv).  All arrays are host memory; the library copies them to the
 * device, runs the whole iteration there and copies the results back.
 *   uplo      'F' full, 'L' lower or 'U' upper triangle stored (Sec. 4.1)
 *   n         order of A and B (> 0)
 *   a, ia, ja CSR of A; ia[0] is the index base (1 as in the guide, or 0);
 *             nnz = ia[n] - ia[0]
 *   b, ib, jb CSR of B in the same storage and base, or all NULL for B = I
 *   fpm       parameters (in/out: fpm(60))
 *   emin,emax search interval
 *   m0        in: subspace size (1..n); out: live subspace size
 *   e         [m0] out: e[0..M-1] eigenvalues inside [emin,emax] ascending,
 *             then the outside Ritz values ascending
 *   x         [n*m0] column-major: in: start subspace if fpm(5)=1;
 *             out: B-orthonormal eigenvectors matching e
 *   m         out: number of eigenvalues found in the interval
 *   res       [m0] out: ||A x - e B x|| / ||alpha B x||, alpha = max(|emin|,|emax|)
 *   epsout    out: relative trace change of the last loop
 *   loop      out: refinement loops done
 *   info      out: as the return value
 * One-pass modes (guide Sec. 3.1, fpm(14); the guide cites Di Napoli, Polizzi
 * and Saad for the estimate): the M0 columns of the start block (X when
 * fpm(5)=1, else seeded normal random vectors) go through one contour pass
 * Q = sum_e Re(w_e (z_e B - A)^{-1} B Y) and no Rayleigh-Ritz step follows.
 * fpm(14)=1 returns Q in x (info 4).  fpm(14)=2 returns in m the nearest
 * integer to the estimate (1/M0) sum_j y_j^T Q_j of trace(rho(B^{-1}A)), the
 * number of eigenvalues inside the contour (rho ~ 1 inside, ~ 0 far
 * outside), with e[0] = the estimate and e[1] = its standard error (sample
 * standard deviation / sqrt(M0), M0 >= 2); x is not changed (info 5).
 * fpm(40) must be 0 here (-> 140); feast_scsr_extreme takes +-1. */
int feast_scsr_solve(char uplo, int n, const double* a, const int* ia, const int* ja, const double* b,
                     const int* ib, const int* jb, int* fpm, double emin, double emax, int* m0, double* e,
                     double* x, int* m, double* res, double* epsout, int* loop, int* info);

/* Expert variant with custom integration nodes (guide Sec. 4.3 "Contour
 * Customization": the "x" routines take the nodes and weights of a
 * user-designed half contour for Hermitian problems).  Arguments as
 * feast_scsr_solve, plus zne, wne: host arrays of 2*fpm(2) doubles,
 * (re, im) interleaved, replacing the rule of fpm(16)/fpm(18); the filter is
 * rho(lambda) = sum_e Re(wne_e / (zne_e - lambda)), the convention of
 * feast_contour_nodes (whose output reproduces the built-in rule).  Every
 * node must lie strictly in the upper half plane; emin/emax still select the
 * eigenvalues reported inside and scale the residuals.  -120 for missing or
 * invalid nodes. */
int feast_scsr_solve_x(char uplo, int n, const double* a, const int* ia, const int* ja, const double* b,
                       const int* ib, const int* jb, int* fpm, double emin, double emax, int* m0, double* e,
                       double* x, int* m, double* res, double* epsout, int* loop, int* info, const double* zne,
                       const double* wne);

/* Extreme-eigenvalue mode (guide Sec. 3.1, fpm(40) = -1 / +1, and Sec. 3.2:
 * the sparse drivers search the M0/2 lowest or largest eigenpairs and return
 * the search interval).  Arguments as feast_scsr_solve, except:
 *   fpm(40)   -1 lowest, +1 largest (anything else -> 140); fpm(14) must be 0
 *   emin,emax host, out: an interval holding exactly the k = M0/2 wanted
 *             eigenvalues (ignored on entry)
 *   m0        in: 2k (2..n); out: live subspace size
 *   e, x, res the k wanted pairs first (e ascending), then the other Ritz pairs
 *   m         out: k
 * The guide does not give the search; this library's: Gershgorin bounds of
 * the pencil (of A for B = I, of D^{-1/2} A D^{-1/2} for B = D diagonal, else
 * A's bounds divided by B's, which must be positive), an interval grown from
 * the low (high) end guided by stochastic counts (fpm(14)=2 with min(M0, 32)
 * probes, seed fpm(52)) until it holds about 1.15k..1.5k eigenvalues, then
 * normal FEAST runs with M0 = 2k on it, widened or narrowed and restarted
 * from the current Ritz vectors until at least k eigenvalues converge inside.
 * Returns 0 (or 2 if the last run did not converge within fpm(4) loops), 7
 * when no interval could be found, or the error codes above; -110/-111 for
 * NULL emin/emax. */
int feast_scsr_extreme(char uplo, int n, const double* a, const int* ia, const int* ja, const double* b,
                       const int* ib, const int* jb, int* fpm, double* emin, double* emax, int* m0, double* e,
                       double* x, int* m, double* res, double* epsout, int* loop, int* info);

/* One problem of a batch (host memory, caller-owned).  CSR in full storage,
 * base ia[0] in {0,1}; b/ib/jb all NULL for B = I (then for every problem of
 * the batch).  x0: column-major n x m0 start subspace, or NULL for a random
 * block.  1 <= m0 <= min(n, 128). */
typedef struct feast_problem {
    int n;
    const double* a;
    const int* ia;
    const int* ja;
    const double* b;
    const int* ib;
    const int* jb;
    double emin, emax;
    int m0;
    const double* x0;
} feast_problem;

/* Result of one problem (host memory, caller-allocated arrays): e[m0],
 * x[n*m0] (column-major eigenvectors), res[m0]; info as in the guide's info
 * table; m eigenvalues found in the interval; loop refinement loops; m0 the
 * live subspace size; epsout the relative trace change. */
typedef struct feast_result {
    int info, m, loop, m0;
    double epsout;
    double* e;
    double* x;
    double* res;
} feast_result;

/* Many independent problems of uneven size and interval solved together (the
 * guide's first level of parallelism, Sec. 1.1: separate search intervals).
 * One set of filter launches serves all unfinished problems; the COCG steps
 * and the batched Rayleigh-Ritz sequence replay as captured CUDA graphs; the
 * rows per work item of the gathering step are picked by timing a few
 * choices on the batch (cached per size class) unless fpm(51) sets them.
 * The contour nodes come from fpm(2), fpm(18) and each problem's interval;
 * fpm(50) defaults to one node per batch.  Each problem starts with a
 * Rayleigh-Ritz step on its start block.  Returns 0 when every problem ran
 * (see out[p].info), -101..-104 for a bad argument (-102: problem p invalid,
 * its out[p].info says why, or some problems have B and others not), -4 on a
 * CUDA error. */
int feast_scsr_solve_batched(int np, const feast_problem* probs, int* fpm, feast_result* out);

/* Device workspace, in bytes, that feast_scsr_solve_dev needs for this
 * problem size and these parameters (fpm(2), fpm(42), fpm(50), fpm(51)). */
size_t feast_scsr_workspace_bytes(int n, int nnz_a, int nnz_b, int m0, const int* fpm);

/* Same as feast_scsr_solve with the matrices and X already on the device.
 * d_ia/d_ja/d_a: 0-based CSR of A in full storage (device); d_ib/d_jb/d_b the
 * same for B or NULL for B = I; d_x: device, column-major n x m0, in/out as x
 * above.  e, res and the scalars are host memory.  d_work: device workspace of
 * at least feast_scsr_workspace_bytes(...) bytes, 256-byte aligned; the
 * library allocates nothing.  Work is enqueued on stream; the call returns
 * once the results are written.  Argument errors as above; the CSR is not
 * re-validated (use feast_scsr_solve for untrusted input). */
int feast_scsr_solve_dev(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                         const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double emin,
                         double emax, int* m0, double* e, double* d_x, int* m, double* res,
                         double* epsout, int* loop, int* info, void* d_work, size_t work_bytes,
                         void* stream);

/* Complex Hermitian problems A x = lambda B x (the guide's zfeast_hcsr{ev,gv},
 * Sec. 3.2 "FEAST Hermitian"; algorithm of Sec. 1.1).  A Hermitian, B
 * Hermitian positive definite or absent (B = I).  Arguments as
 * feast_scsr_solve, except that a and b hold nnz complex values as
 * interleaved (real, imaginary) doubles, 'L' / 'U' storage mirrors an entry
 * a_ij as conj(a_ij), and x is column-major n x m0 complex (interleaved,
 * 2 n m0 doubles).  The eigenvalues are real.  Both halves of the contour are
 * solved: BiCG on z_e B - A with the conjugate-shift shadow system, so every
 * node gives G(z_e) and G(conj z_e) in one run; Rayleigh-Ritz in complex FP64.
 * fpm as for the real driver (fpm(2), (3), (4), (5), (6), (16) rules 0-2,
 * (18), (42), (45), (46), (50) node batch <= 32, (52) seed), except that
 * fpm(14) and fpm(40) must be 0 (info 114, 140); m0 <= 1024 (else 201).
 * Device memory (CSR copies, X and the workspace) is allocated per call.
 * Returns info. */
int feast_hcsr_solve(char uplo, int n, const double* a, const int* ia, const int* ja, const double* b,
                     const int* ib, const int* jb, int* fpm, double emin, double emax, int* m0, double* e,
                     double* x, int* m, double* res, double* epsout, int* loop, int* info);

/* feast_hcsr_solve with the matrices and X on the device: d_ia/d_ja 0-based
 * full-storage CSR, d_a / d_b nnz complex doubles (interleaved), d_ib NULL for
 * B = I, d_x column-major n x m0 complex (in/out).  e, res and the scalars
 * are host memory.  d_work: a caller-owned device workspace of work_bytes >=
 * feast_hcsr_workspace_bytes(...) bytes (256-byte aligned), from which every
 * device buffer of the solve is carved, so the call allocates nothing; or
 * NULL, and the library allocates the workspace for the call (cudaMalloc) and
 * frees it before returning.  A workspace that is too small gives -120.  Work
 * is enqueued on stream (NULL: the default stream) and the call returns once
 * the results are written.  The CSR is not re-validated. */
int feast_hcsr_solve_dev(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                         const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double emin,
                         double emax, int* m0, double* e, double* d_x, int* m, double* res,
                         double* epsout, int* loop, int* info, void* d_work, size_t work_bytes,
                         void* stream);

/* Device workspace, in bytes, that feast_hcsr_solve_dev needs for this
 * problem size and these parameters (fpm(2), fpm(42), fpm(50)); 0 for
 * invalid sizes. */
size_t feast_hcsr_workspace_bytes(int n, int nnz_a, int nnz_b, int m0, const int* fpm);

/* feast_scsr_solve_dev with custom nodes zne, wne (host, as for
 * feast_scsr_solve_x); -124 for missing or invalid nodes. */
int feast_scsr_solve_dev_x(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                           const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double emin, double emax,
                           int* m0, double* e, double* d_x, int* m, double* res, double* epsout, int* loop,
                           int* info, void* d_work, size_t work_bytes, void* stream, const double* zne,
                           const double* wne);

/* feast_scsr_extreme with the matrices and X on the device, arguments as
 * feast_scsr_solve_dev; emin and emax are host pointers (out).  d_work: at
 * least feast_scsr_workspace_bytes(...) bytes for this fpm (fpm(40) != 0 adds
 * room for -A, diag(B) and the Gershgorin partials). */
int feast_scsr_extreme_dev(int n, int nnz_a, const int* d_ia, const int* d_ja, const double* d_a, int nnz_b,
                           const int* d_ib, const int* d_jb, const double* d_b, int* fpm, double* emin,
                           double* emax, int* m0, double* e, double* d_x, int* m, double* res, double* epsout,
                           int* loop, int* info, void* d_work, size_t work_bytes, void* stream);

/* ---------------------------------------------------------------- kernels
 * Device-pointer entry points of the individual steps, for testing and for
 * callers that assemble their own iteration.  Each enqueues on stream and
 * returns 0 or -4 (CUDA error) / -(100+i) (bad argument i); those that need
 * scratch allocate it with cudaMallocAsync on the stream. */

/* Layout of the filter's complex block vectors for nb contour nodes solved
 * at once in precision fp64 (0: complex float, 1: complex double): a tile
 * of W complex values per row holds mt subspace columns x nbp node lanes,
 * node fastest; element (node e, column j, row i) sits at complex index
 * (g*n + i)*W + (j % mt)*nbp + e with g = j / mt.  Returns 0. */
int feast_filter_layout(int nb, int fp64, int* W, int* nbp, int* mt);

/* Batched complex-shifted CSR SpMM (the inner product of every COCG step):
 * V_e = (z_e B - A) P_e for nb nodes and m columns in one launch, in the
 * layout of feast_filter_layout.  z: host, 2*nb doubles (re, im).  A, B:
 * 0-based device CSR with FP64 values, rounded to float when fp64 = 0 (as
 * the mixed-precision solver does); B may be NULL (identity).  P, V: device
 * complex float (fp64 = 0) or complex double (fp64 = 1) tiles. */
int feast_shifted_spmm_dev(int n, int nnz_a, const int* ia, const int* ja, const double* a, int nnz_b,
                           const int* ib, const int* jb, const double* b, int nb, const double* z, int m,
                           int fp64, const void* P, void* V, void* stream);

/* One filter pass over all ne nodes (guide Sec. 1.1 quadrature; Sec. 3.1
 * residual inverse form):
 *   rii = 0:  Q = sum_e Re(w_e Y_e),                  (z_e B - A) Y_e = R
 *   rii = 1:  Q = X diag(rho(lam)) + sum_e Re(w_e/(z_e - lam_j) Y_e[:,j]),
 *             rho(l) = sum_e Re(w_e/(z_e - l))
 * with the shifted systems solved by column-batched COCG to relative residual
 * 10^-fpm(45) or fpm(46) steps, in precision fpm(42) (1: complex float,
 * 0: complex double).  A/B: 0-based device CSR with FP64 values (B NULL = I);
 * R, X, Q: device row-major n x m (R(i,j) at R[i*m + j]); lam: device [m];
 * nodes from fpm(2), fpm(18), emin, emax.  *iters (host, may be NULL): COCG
 * steps taken (max over columns, summed over node batches). */
int feast_filter_dev(int n, int nnz_a, const int* ia, const int* ja, const double* a, int nnz_b, const int* ib,
                     const int* jb, const double* b, int m, const double* R, const double* X,
                     const double* lam, int rii, const int* fpm, double emin, double emax, double* Q,
                     int* iters, void* stream);

/* C = X^T Y (m x m, row-major), X and Y device row-major n x m, FP64; only
 * the upper triangle is computed and the result is that triangle mirrored,
 * C[i][j] = (X^T Y)[min(i,j)][max(i,j)] (the Rayleigh-Ritz matrices Q^T A Q
 * and Q^T B Q are symmetric up to rounding, and this is their symmetric
 * form). */
int feast_gram_dev(int n, int m, const double* X, const double* Y, double* C, void* stream);

/* Allocation-free variant of feast_gram_dev (the paper has no counterpart:
 * it is a library convenience).  Same arguments and result, but the split-K
 * partial sums live in a fixed 16 MiB array that the library keeps in the
 * device memory of every GPU that loads it, so the call needs no cudaMalloc,
 * no cudaMallocAsync and no caller workspace.  It serves callers that cannot
 * allocate device memory at the point of the call, e.g. code working inside
 * a memory pool owned by another runtime, code that must avoid the implicit
 * synchronisation of cudaMalloc/cudaFree, or an interface with no room for a
 * workspace argument.
 *   - Limit: m*m <= 2097152 (m <= 1448); larger m returns -102 with a message
 *     in feast_last_error().  n > 0, else -101.  CUDA failures return -4.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before capturing a stream into a CUDA graph.
 *   - All calls share the one array and it keeps the last call's partial sums;
 *     each call overwrites every partial it reads, so nothing needs clearing.
 *     Calls whose execution overlaps on the GPU (different streams, or host
 *     threads not ordered by the caller) race on the array: serialise them.
 *   - Enqueues on stream and returns after C is written. */
int feast_gram_noalloc_dev(int n, int m, const double* X, const double* Y, double* C, void* stream);

/* The same contraction C = X^T Y (upper triangle mirrored) computed from
 * exact products of BF16 integer slices on the tensor cores (Ozaki et al.'s
 * error-free splitting: 8 slices of 7 bits per value under a power-of-two
 * column scale; products accumulated exactly in FP32 for 256 rows at a time,
 * then in FP64), the arithmetic of the solvers' projections A_Q = Q^T A Q,
 * B_Q = Q^T B Q when fpm(54) = 0 (Sec. 1.1's reduced problem, FP64 accuracy:
 * the truncation error of an element is below 2^-55 max|X[:,a]| max|Y[:,b]|
 * per row).  Device row-major n x m X, Y; C m x m.  Returns 0, -101 n <= 0,
 * -102 m <= 0, -4 on a CUDA error. */
int feast_gram_oz_dev(int n, int m, const double* X, const double* Y, double* C, void* stream);

/* C = A V: A device row-major n x m, V device row-major m x k, C n x k, FP64. */
int feast_gemm_dev(int n, int m, int k, const double* A, const double* V, double* C, void* stream);

/* C = A V as feast_gemm_dev, from exact BF16 slice products on the tensor
 * cores under a power-of-two scale per row of A and per column of V (the
 * arithmetic of the Ritz vectors X = Q V when fpm(54) = 0; FP64 accuracy:
 * truncation below 2^-55 max|A[i,:]| max|V[:,c]| per term).  Same arguments
 * and return codes as feast_gemm_dev. */
int feast_gemm_oz_dev(int n, int m, int k, const double* A, const double* V, double* C, void* stream);

/* Symmetric eigen-decomposition (cyclic Jacobi) of the device m x m matrix A
 * (row-major, destroyed): lam ascending, V row-major with eigenvectors in
 * columns.  *sweeps (host, may be NULL).  Returns 0, or -3 on no convergence. */
int feast_sym_eig_dev(int m, double* A, double* lam, double* V, int* sweeps, void* stream);

/* Reduced generalized problem A_q v = lambda B_q v (device row-major m x m):
 * lam ascending with *mk (host) live values first (directions where B_q is
 * numerically singular are dropped and sort last with values >= 1e299); V
 * row-major m x m with V^T B_q V = I on the live columns.  Returns 0, or -3. */
int feast_reduced_eig_dev(int m, const double* Aq, const double* Bq, double* lam, double* V, int* mk,
                          void* stream);

/* Residual block R = A X - B X diag(lam) (device row-major n x m) and
 * res[j] = ||R_j|| / (alpha ||B x_j||) (device [m]); A/B 0-based device CSR
 * (B NULL = I). */
int feast_residual_dev(int n, const int* ia, const int* ja, const double* a, const int* ib, const int* jb,
                       const double* b, int m, const double* X, const double* lam, double alpha, double* R,
                       double* res, void* stream);

/* Gradient of L = sum_k g_k lambda_k over the stored entries of a CSR
 * pattern: grad[p] = sum_k w_k x_k[i_p] x_k[j_p] with w_k = g_k for the
 * entries of A and w_k = -g_k lambda_k for those of B (first-order
 * perturbation of a simple eigenpair with x^T B x = 1).  Device: ia/ja
 * (0-based), X row-major n x m, w [m], grad [nnz].  m <= 2048. */
int feast_eig_grad_dev(int n, const int* ia, const int* ja, int m, const double* X, const double* w,
                       double* grad, void* stream);

/* Time limit of the library's bounded device waits (a library setting; the
 * guide has no counterpart).  The reduced eigensolver runs its Jacobi rounds
 * in one cooperative launch whose CTAs meet at a grid barrier every round;
 * a CTA that spins there for more than `cycles` SM clock cycles sets an error
 * flag that makes every CTA of the launch return, and the call reports the
 * failure (-3 from the solvers and the reduced-eigensolver entry points) with the
 * context still usable.  The COCG gathering step waits on an mbarrier for the
 * bulk copies that stage its rows; a CTA whose wait exceeds the limit sets an
 * error flag, lets its copies in flight land (waiting up to about a second
 * more) and returns, and the solver reports -4 (message in feast_last_error).
 * Default 4e9 cycles (about two seconds at 2 GHz); cycles < 1 restores the
 * default.  Applies to launches issued after the call, process-wide.  Returns
 * the previous limit. */
long long feast_set_wait_limit(long long cycles);

/* Gradient of an eigenvalue loss over the stored entries of A and B, host
 * buffers (the boundary's counterpart of the device feast_eig_grad_dev; the
 * guide has no differentiation interface: this is first-order perturbation
 * theory of a simple eigenpair, not a passage of the guide).  For
 * L = sum_k g_k lambda_k and eigenpairs of A x = lambda B x with x^T B x = 1:
 *   grad_a[p] = sum_k g_k x_k[i_p] x_k[j_p]
 *   grad_b[p] = -sum_k g_k lambda_k x_k[i_p] x_k[j_p]
 * per stored entry p = (i_p, j_p) of the patterns as passed.
 *   uplo      'F': full storage, one derivative per stored entry (perturbing a
 *             symmetric pair (i,j),(j,i) moves L by the sum of both);
 *             'L'/'U': one triangle stored, as for feast_scsr_solve, so an
 *             off-diagonal value stands for both entries and gets twice the
 *             entry-wise derivative
 *   n         order (>= 1)
 *   ia, ja    A's CSR pattern, base ia[0] in {0,1} (values are not needed)
 *   ib, jb    B's CSR pattern, or both NULL for B = I (grad_b unused)
 *   m         eigenpairs in the loss, 0 <= m <= 2048
 *   x         [n*m] column-major eigenvectors (B-orthonormal, as returned by
 *             feast_scsr_solve in its first m columns)
 *   e         [m] eigenvalues (needed only with B)
 *   g         [m] loss weights
 *   grad_a    [nnz(A)] out;  grad_b  [nnz(B)] out
 * Every array is caller-owned host memory; the library copies to the device,
 * runs the SDDMM kernel and copies the gradients back (synchronous).
 * Eigenvalues in the loss must be simple.  Returns 0; 202 for n <= 0;
 * -101 bad uplo; -(100+i) for a bad i-th argument (pattern out of range or
 * outside the stored triangle, NULL array, m out of range); -4 on a CUDA error
 * (message in feast_last_error). */
int feast_scsr_grad(char uplo, int n, const int* ia, const int* ja, const int* ib, const int* jb, int m,
                    const double* x, const double* e, const double* g, double* grad_a, double* grad_b);

#ifdef __cplusplus
}
#endif

#endif /* FEAST_GB300_H */
