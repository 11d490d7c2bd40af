// rb_eim.cu -- empirical interpolation (EI) nodes of a basis and out-of-sample
// validation (the software of Sec. 6.1: "QR+DEIM").
//
// Nodes: the greedy EIM / DEIM rule -- p_1 = argmax |q_1|; p_i = argmax over
// the grid points not yet chosen of the residual r_i of q_i after
// interpolation on p_1..p_{i-1} with q_1..q_{i-1}.  That residual is column i
// of the Schur complement of Gaussian elimination with partial pivoting on the
// N x k matrix of basis vectors, so the nodes come from a right-looking
// elimination: step i picks p_i on column i (a grid argmax, ties to the lower
// index) and removes column i from the later columns with the multipliers
// W(p_i, l) / W(p_i, i).  Afterwards column m of the working copy is r_m, and
// with L = R(P, :) (lower triangular, L[n][m] = r_m(p_n)) the interpolant is
// B = Q V^{-1} = R L^{-1} (V = Q(P, :) = L U for a unit upper U), one
// triangular solve per grid point.  FP64 throughout.
//
// Validation: for a snapshot t with coefficients c = Q^H t, the projection
// error is ||t||^2 - ||c||^2 (Eq. (Residual)) and, since I[.] reproduces the
// span of Q and t - Q c is orthogonal to it,
//   ||t - I[t]||^2 = ||t - Q c||^2 + ||V^{-1} t(P) - c||^2,
// so the interpolation error needs only the k values t(P) and V^{-1}.
#include <climits>

#include "rb_internal.cuh"

namespace rbk {

constexpr int EI_THREADS = 256;

// Step i: p_i = argmax over free x of |W[:, i]|^2 (ties to the lower x).  The
// last block records the node, marks it taken and forms the multipliers
// mult[l] = W[p, l] / W[p, i] of the later columns; when the residual
// vanished on every free point it raises *flag and the multipliers are zero.
__global__ void __launch_bounds__(EI_THREADS) k_eim_pick(const double2 *__restrict__ W, long long N, int k, int i,
                                                         unsigned char *__restrict__ taken, double *__restrict__ pv,
                                                         long long *__restrict__ pi, unsigned int *__restrict__ ticket,
                                                         long long *__restrict__ nodes, double2 *__restrict__ mult,
                                                         int *__restrict__ flag) {
    double best = -1.0;
    long long bi = LLONG_MAX;
    const double2 *w = W + (long long)i * N;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
        if (taken[x]) continue;
        const double2 v = w[x];
        const double a = v.x * v.x + v.y * v.y;
        if (better(a, x, best, bi)) {
            best = a;
            bi = x;
        }
    }
    block_best(best, bi);
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = best;
        pi[blockIdx.x] = bi;
    }
    if (!last_block(ticket)) return;
    double b2 = -1.0;
    long long i2 = LLONG_MAX;
    for (int u = threadIdx.x; u < (int)gridDim.x; u += blockDim.x)
        if (better(pv[u], pi[u], b2, i2)) {
            b2 = pv[u];
            i2 = pi[u];
        }
    block_best(b2, i2);
    __shared__ long long sp;
    if (threadIdx.x == 0) {
        *ticket = 0;
        if (i2 < 0 || i2 >= N) i2 = 0;  // only when every point is taken (k > N is rejected on the host)
        if (!(b2 > 0.0)) *flag = 1;
        nodes[i] = i2;
        taken[i2] = 1;
        sp = i2;
    }
    __syncthreads();
    const long long p = sp;
    const double2 piv = W[(long long)i * N + p];
    const double d = piv.x * piv.x + piv.y * piv.y;
    for (int l = i + 1 + threadIdx.x; l < k; l += blockDim.x) {
        const double2 a = W[(long long)l * N + p];
        mult[l] = d > 0.0 ? make_double2((a.x * piv.x + a.y * piv.y) / d, (a.y * piv.x - a.x * piv.y) / d)
                          : make_double2(0.0, 0.0);
    }
}

// Step i: W[:, l] -= W[:, i] mult[l] for the later columns l = i + 1 + y; the
// pivot row becomes exactly zero.
__global__ void __launch_bounds__(EI_THREADS) k_eim_update(double2 *__restrict__ W, long long N, int i,
                                                           const long long *__restrict__ nodes,
                                                           const double2 *__restrict__ mult) {
    const int l = i + 1 + blockIdx.y;
    const long long p = nodes[i];
    const double2 m = mult[l];
    double2 *wl = W + (long long)l * N;
    const double2 *wi = W + (long long)i * N;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
        if (x == p) {
            wl[x] = make_double2(0.0, 0.0);
            continue;
        }
        const double2 a = wi[x];
        double2 b = wl[x];
        b.x = fma(-a.x, m.x, fma(a.y, m.y, b.x));
        b.y = fma(-a.x, m.y, fma(-a.y, m.x, b.y));
        wl[x] = b;
    }
}

// L[n][m] = r_m(p_n) (zero above the diagonal) and, when asked, V[n][m] = q_m(p_n).
__global__ void k_eim_gather(const double2 *__restrict__ W, long long N, const double2 *__restrict__ Q, long long ldQ,
                             int k, const long long *__restrict__ nodes, double2 *__restrict__ L,
                             double2 *__restrict__ V) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < (long long)k * k;
         u += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(u / k), m = (int)(u % k);
        const long long p = nodes[n];
        L[u] = m <= n ? W[(long long)m * N + p] : make_double2(0.0, 0.0);
        if (V) V[u] = Q[(long long)m * ldQ + p];
    }
}

// B = R L^{-1}: for every grid point x, b L = r(x), solved from the last
// column down: b_m = (r_m(x) - sum_{n > m} b_n L[n][m]) / L[m][m].
__global__ void __launch_bounds__(EI_THREADS) k_eim_interpolant(const double2 *__restrict__ W, long long N, int k,
                                                                const double2 *__restrict__ L, double2 *__restrict__ B,
                                                                long long ldB) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
        for (int m = k - 1; m >= 0; m--) {
            double2 b = W[(long long)m * N + x];
            for (int n = m + 1; n < k; n++) {
                const double2 bn = B[(long long)n * ldB + x], l = L[n * k + m];
                b.x = fma(-bn.x, l.x, fma(bn.y, l.y, b.x));
                b.y = fma(-bn.x, l.y, fma(-bn.y, l.x, b.y));
            }
            const double2 d = L[m * k + m];
            const double dd = d.x * d.x + d.y * d.y;
            B[(long long)m * ldB + x] = make_double2((b.x * d.x + b.y * d.y) / dd, (b.y * d.x - b.x * d.y) / dd);
        }
    }
}

size_t eim_workspace(long long N, int k) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const long long nb = eim_blocks(N);
    return up((size_t)N * k * 16) + up((size_t)k * k * 16) + up((size_t)k * 16) + up((size_t)N) + up((size_t)nb * 8) * 2 +
           up(64);
}

long long eim_blocks(long long N) {
    long long nb = (N + EI_THREADS - 1) / EI_THREADS;
    return nb < 1 ? 1 : (nb > 1024 ? 1024 : nb);
}

cudaError_t launch_eim(const double2 *Q, long long N, int k, long long ldQ, void *ws, long long *nodes, double2 *V,
                       double2 *B, long long ldB, int *flag, cudaStream_t s) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const long long nb = eim_blocks(N);
    char *w = (char *)ws;
    double2 *W = (double2 *)w;
    w += up((size_t)N * k * 16);
    double2 *L = (double2 *)w;
    w += up((size_t)k * k * 16);
    double2 *mult = (double2 *)w;
    w += up((size_t)k * 16);
    unsigned char *taken = (unsigned char *)w;
    w += up((size_t)N);
    double *pv = (double *)w;
    w += up((size_t)nb * 8);
    long long *pi = (long long *)w;
    w += up((size_t)nb * 8);
    unsigned int *ticket = (unsigned int *)w;
    cudaError_t e;
    if ((e = cudaMemcpy2DAsync(W, (size_t)N * 16, Q, (size_t)ldQ * 16, (size_t)N * 16, (size_t)k,
                               cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(taken, 0, (size_t)N, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(ticket, 0, 64, s)) != cudaSuccess)
        return e;
    for (int i = 0; i < k; i++) {
        k_eim_pick<<<(unsigned)nb, EI_THREADS, 0, s>>>(W, N, k, i, taken, pv, pi, ticket, nodes, mult, flag);
        if (i + 1 < k) k_eim_update<<<dim3((unsigned)nb, (unsigned)(k - 1 - i)), EI_THREADS, 0, s>>>(W, N, i, nodes, mult);
    }
    const long long gg = ((long long)k * k + 255) / 256;
    k_eim_gather<<<(unsigned)(gg < 1024 ? gg : 1024), 256, 0, s>>>(W, N, Q, ldQ, k, nodes, L, V);
    if (B) k_eim_interpolant<<<(unsigned)nb, EI_THREADS, 0, s>>>(W, N, k, L, B, ldB);
    return cudaGetLastError();
}

// ------------------------------------------------------------- validation
// One warp per snapshot t_j: ||t_j||^2 (FP64), ||c_j||^2 from the stored
// coefficients C[l * ldC + j], err_proj = max(||t||^2 - ||c||^2, 0); with
// nodes, y = Vinv t(P) - c and err_eim = err_proj + ||y||^2.  t(P) is staged
// per warp in shared memory (k values).
__global__ void __launch_bounds__(128) k_validate(const double2 *__restrict__ T, long long N, long long Mt, long long ldT,
                                                  const double2 *__restrict__ C, long long ldC, int k,
                                                  const long long *__restrict__ nodes,
                                                  const double2 *__restrict__ Vinv, double *__restrict__ err_proj,
                                                  double *__restrict__ err_eim) {
    extern __shared__ double2 tp[];  // 4 warps x k
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    double2 *mytp = tp + (long long)wl * k;
    const long long nw = (long long)gridDim.x * 4;
    for (long long j = blockIdx.x * 4LL + wl; j < Mt; j += nw) {
        const double2 *t = T + j * ldT;
        double s = 0.0;
        for (long long x = lane; x < N; x += 32) {
            const double2 v = t[x];
            s = fma(v.x, v.x, fma(v.y, v.y, s));
        }
        double cs = 0.0;
        for (int l = lane; l < k; l += 32) {
            const double2 c = C[(long long)l * ldC + j];
            cs = fma(c.x, c.x, fma(c.y, c.y, cs));
        }
        s = warp_sum(s);
        cs = warp_sum(cs);
        const double ep = s - cs > 0.0 ? s - cs : 0.0;
        if (lane == 0) err_proj[j] = ep;
        if (!err_eim) continue;
        for (int n = lane; n < k; n += 32) mytp[n] = t[nodes[n]];
        __syncwarp();
        double ys = 0.0;
        for (int m = lane; m < k; m += 32) {
            double2 y = C[(long long)m * ldC + j];
            y.x = -y.x;
            y.y = -y.y;
            for (int n = 0; n < k; n++) {
                const double2 a = Vinv[(long long)m * k + n], b = mytp[n];
                y.x = fma(a.x, b.x, fma(-a.y, b.y, y.x));
                y.y = fma(a.x, b.y, fma(a.y, b.x, y.y));
            }
            ys = fma(y.x, y.x, fma(y.y, y.y, ys));
        }
        ys = warp_sum(ys);
        if (lane == 0) err_eim[j] = ep + ys;
        __syncwarp();
    }
}

cudaError_t launch_validate(const double2 *T, long long N, long long Mt, long long ldT, const double2 *C, long long ldC,
                            int k, const long long *nodes, const double2 *Vinv, double *err_proj, double *err_eim,
                            cudaStream_t s) {
    if (Mt <= 0) return cudaSuccess;
    const size_t sm = (size_t)4 * (k > 0 ? k : 1) * 16;
    cudaError_t e;
    if (sm > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_validate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
        return e;
    long long g = (Mt + 3) / 4;
    if (g > 4096) g = 4096;
    k_validate<<<(unsigned)g, 128, sm, s>>>(T, N, Mt, ldT, C, ldC, k, nodes, Vinv, err_proj, err_eim);
    return cudaGetLastError();
}

}  // namespace rbk
