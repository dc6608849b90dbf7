// One-CTA Cholesky factorization and triangular inverse used by the reduced
// generalized eigenproblem A_Q v = lambda B_Q v of the Rayleigh-Ritz step
// (FEAST v4.0 guide, Sec. 1.1; the guide's dense reduced solvers are the
// LAPACK sygv family, whose first step is B = L L^T).
//
// With B~ = L L^T and X = L^{-1}, S = D X^T satisfies S^T B_Q S = I for the
// diagonal scaling D, so the generalized problem turns into the standard one
// S^T A_Q S w = lambda w.  When the filtered subspace is nearly B-orthogonal
// (every loop after the first few), B~ is close to I, L is close to I and
// S^T A_Q S stays close to diagonal, so the Jacobi sweeps that follow converge
// in a few sweeps.
#pragma once

namespace feast {

static constexpr double kCholCondMax = 1e8;  // accepted bound on ||L^{-1}||_F^2

// All threads of the CTA call this.  M: m x m row-major holding the symmetric
// positive definite B~ (lower triangle read).  On return true: lower triangle
// of M (with the diagonal) = L, xd[i] = 1 / L_ii, strict upper triangle of M =
// the strict upper triangle of X^T (M[c][i] = X[i][c], c < i).  Returns false
// when a pivot is not positive or ||X||_F^2 > kCholCondMax; M is then
// partially overwritten.  cj: m doubles of scratch; red: blockDim.x / 32
// doubles of shared scratch.  Right-looking factorization: two CTA barriers
// per column.  The inverse needs none: warp w owns the columns c = w, w + nw,
// ... of X and runs the forward substitution
// X[i][c] = -(1/L_ii) sum_{c<=k<i} L[i][k] X[k][c] down its columns.
__device__ inline bool cta_chol_inv(int m, double* M, double* xd, double* cj, double* red)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int j = 0; j < m; ++j) {
        const double d = M[(size_t)j * m + j];
        if (!(d > 0.0)) return false;  // same value in every thread: uniform exit
        const double l = sqrt(d);
        for (int i = j + 1 + tid; i < m; i += nt) {
            const double v = M[(size_t)i * m + j] / l;
            M[(size_t)i * m + j] = v;
            cj[i] = v;
        }
        if (tid == 0) xd[j] = l;
        __syncthreads();
        for (int i = j + 1 + warp; i < m; i += nw) {
            const double ci = cj[i];
            for (int k = j + 1 + lane; k <= i; k += 32) M[(size_t)i * m + k] -= ci * cj[k];
        }
        __syncthreads();
    }
    for (int i = tid; i < m; i += nt) {
        const double l = xd[i];
        M[(size_t)i * m + i] = l;
        xd[i] = 1.0 / l;
    }
    __syncthreads();
    double nrm = 0.0;
    for (int c = warp; c < m; c += nw) {
        const double xc = xd[c];
        if (lane == 0) nrm += xc * xc;
        for (int i = c + 1; i < m; ++i) {
            double s = 0.0;
            for (int k = c + lane; k < i; k += 32)
                s = fma(M[(size_t)i * m + k], k == c ? xc : M[(size_t)c * m + k], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const double v = -s * xd[i];
            if (lane == 0) {
                M[(size_t)c * m + i] = v;
                nrm += v * v;
            }
            __syncwarp();
        }
    }
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (lane == 0) red[warp] = nrm;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < nw; ++w) tot += red[w];
    __syncthreads();
    return tot <= kCholCondMax;
}

}  // namespace feast
