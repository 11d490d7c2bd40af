// rb_project.cu -- projection coefficients C = Q^H X (Sec. 2: a column is
// represented by its orthogonal projection onto the span of the basis).
//
// First form: a shared-memory tiled complex GEMM in plain FP64.  Each block
// computes a TL x TJ tile of C, staging TK rows of Q and X per step.
#include "rb_internal.cuh"

namespace rbk {

constexpr int PJ = 16, PL = 16, PK = 32;

__global__ void __launch_bounds__(PJ *PL) k_project_fp64(const double2 *__restrict__ Q, long long N, int k,
                                                          long long ldQ, const double2 *__restrict__ X,
                                                          long long Mx, long long ldX, double2 *__restrict__ C,
                                                          long long ldC) {
    __shared__ double2 qs[PL][PK + 1];
    __shared__ double2 xs[PJ][PK + 1];
    const int tj = threadIdx.x % PJ, tl = threadIdx.x / PJ;
    const long long j0 = (long long)blockIdx.x * PJ;
    const int l0 = blockIdx.y * PL;
    double re = 0.0, im = 0.0;
    for (long long i0 = 0; i0 < N; i0 += PK) {
        for (int t = threadIdx.x; t < PL * PK; t += PJ * PL) {
            int r = t / PK, c = t % PK;
            long long i = i0 + c;
            qs[r][c] = (l0 + r < k && i < N) ? Q[(long long)(l0 + r) * ldQ + i] : make_double2(0.0, 0.0);
            xs[r][c] = (j0 + r < Mx && i < N) ? X[(j0 + r) * ldX + i] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < PK; c++) {
            double2 a = qs[tl][c], b = xs[tj][c];
            re = fma(a.x, b.x, fma(a.y, b.y, re));
            im = fma(a.x, b.y, fma(-a.y, b.x, im));
        }
        __syncthreads();
    }
    long long j = j0 + tj;
    int l = l0 + tl;
    if (j < Mx && l < k) C[(long long)l * ldC + j] = make_double2(re, im);
}

cudaError_t launch_project(const double2 *Q, long long N, int k, long long ldQ, const double2 *X, long long Mx,
                           long long ldX, double2 *C, long long ldC, cudaStream_t s) {
    if (k <= 0 || Mx <= 0) return cudaSuccess;
    dim3 grid((unsigned)((Mx + PJ - 1) / PJ), (unsigned)((k + PL - 1) / PL));
    k_project_fp64<<<grid, PJ * PL, 0, s>>>(Q, N, k, ldQ, X, Mx, ldX, C, ldC);
    return cudaGetLastError();
}

}  // namespace rbk
