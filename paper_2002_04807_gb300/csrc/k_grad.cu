// Gradient of an eigenvalue loss with respect to the stored CSR values
// (differentiation of the FEAST result; the guide has no counterpart).
// For a simple eigenpair of A x = lambda B x with x^T B x = 1,
// d lambda / d a_ij = x_i x_j and d lambda / d b_ij = -lambda x_i x_j
// (first-order perturbation of a single stored entry).  For the loss
// L = sum_k g_k lambda_k the entry-wise gradient over a CSR pattern is
//   grad[p] = sum_k w_k x_k[i_p] x_k[j_p],  w_k = g_k (for A) or -g_k lambda_k (for B),
// a sampled dense-dense product (SDDMM) over the pattern.
#include "feast_internal.cuh"

namespace feast {

// One warp per row i; Xr is row-major n x m (eigenvectors in columns).
// Weights: w_k = g_k, or w_k = -g_k lambda_k when lam is given (entries of B).
// half: the pattern is one triangle of a symmetric matrix, so a stored
// off-diagonal value stands for both (i, j) and (j, i) and its derivative is
// twice the entry-wise one.
__global__ void __launch_bounds__(256) eig_grad(int n, const int* __restrict__ ia, const int* __restrict__ ja, int m,
                                                const double* __restrict__ Xr, const double* __restrict__ gw,
                                                const double* __restrict__ lam, int half, double* __restrict__ grad)
{
    extern __shared__ double u_sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double* u = u_sm + (size_t)wib * m;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nwarps) {
        for (int k = lane; k < m; k += 32) {
            const double w = lam ? -gw[k] * lam[k] : gw[k];
            u[k] = w * Xr[(size_t)i * m + k];
        }
        __syncwarp();
        for (int p = ia[i]; p < ia[i + 1]; ++p) {
            const int j = ja[p];
            double s = 0.0;
            for (int k = lane; k < m; k += 32) s = fma(u[k], __ldg(Xr + (size_t)j * m + k), s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) grad[p] = (half && j != i) ? 2.0 * s : s;
        }
        __syncwarp();
    }
}

cudaError_t launch_eig_grad(int n, const int* ia, const int* ja, int m, const double* Xr, const double* gw,
                            double* grad, cudaStream_t s, const double* lam, int half)
{
    if (n <= 0) return cudaSuccess;
    if (m <= 0 || m > 2048) return cudaErrorInvalidValue;
    const size_t smem = (size_t)8 * m * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(eig_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    long long blocks = ((long long)n + 7) / 8;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    eig_grad<<<(int)blocks, 256, smem, s>>>(n, ia, ja, m, Xr, gw, lam, half, grad);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace feast
