// rb_recon.cu -- the reconstruction step (Alg. 4, Sec. 5.2.2): the singular
// value decomposition of R(1:j, 1:M) = C = Q_j^H S and the enriched basis
// X_k = Q_j V(:, 1:k).
//
// Only the left factor of C (j x M, j small, M large) is needed, so the SVD is
// taken through the j x j Gram matrix G = C C^H = V Sigma^2 V^H, in two passes:
// pass 1 diagonalises G with Jacobi rotations; pass 2 forms B = V^H C, whose
// rows are already nearly orthogonal, and diagonalises B B^H again.  Pass 1
// alone loses the small singular values to the squaring (relative error
// ~ u sigma_1^2 / sigma_i^2); pass 2 restores relative accuracy (the Jacobi
// method is relatively accurate on a nearly diagonal positive matrix).
//
// Jacobi: cyclic, parallel ("round robin") ordering -- every step rotates
// npad/2 disjoint index pairs at once, left updates of all pairs, a barrier,
// right updates, a barrier.  One block; G and V live in global memory (L1/L2).
// For a pair (p, q) with g = G_pq = |g| e^{i phi}: tau = (G_qq - G_pp) / (2|g|),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c, and
// J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] on columns (p, q); G <- J^H G J,
// V <- V J (the Hermitian form of the symmetric Schur rotation).
//
// All arithmetic is FP64.  Sums run in a fixed order; results are
// deterministic.
#include "rb_internal.cuh"

namespace rbk {

constexpr int RT = 32;   // Gram tile (rows and columns)
constexpr int RTW = 32;  // columns of A per shared-memory step
constexpr long long kGramChunk = 4096;  // columns of A per partial Gram sum

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// Partial Gram tiles: part[chunk][a][b] = sum_{m in chunk} A[a][m] conj(A[b][m])
// for the tile (a0, b0) = (blockIdx.y, blockIdx.z) * RT with a0 <= b0.
// A is j x M, row a at A + a * ldA.  Thread (ty, tx) owns a = a0 + ty and
// b = b0 + 4 tx + e, e < 4.
__global__ void __launch_bounds__(256) k_gram_part(const double2 *__restrict__ A, long long ldA, int j, long long M,
                                                   long long chunk, double2 *__restrict__ part) {
    const int a0 = blockIdx.y * RT, b0 = blockIdx.z * RT;
    if (b0 < a0) return;
    __shared__ double2 sa[RT][RTW + 1], sb[RT][RTW + 1];
    const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;
    const long long m0 = (long long)blockIdx.x * chunk, m1 = m0 + chunk < M ? m0 + chunk : M;
    double2 acc[4];
#pragma unroll
    for (int e = 0; e < 4; e++) acc[e] = make_double2(0.0, 0.0);
    for (long long mt = m0; mt < m1; mt += RTW) {
        for (int u = threadIdx.x; u < RT * RTW; u += blockDim.x) {
            const int r = u / RTW, cc = u % RTW;
            const long long m = mt + cc;
            const bool in = m < m1;
            sa[r][cc] = (in && a0 + r < j) ? A[(long long)(a0 + r) * ldA + m] : make_double2(0.0, 0.0);
            sb[r][cc] = (in && b0 + r < j) ? A[(long long)(b0 + r) * ldA + m] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int cc = 0; cc < RTW; cc++) {
            const double2 x = sa[ty][cc];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const double2 y = sb[4 * tx + e][cc];
                acc[e].x = fma(x.x, y.x, fma(x.y, y.y, acc[e].x));
                acc[e].y = fma(x.y, y.x, fma(-x.x, y.y, acc[e].y));
            }
        }
        __syncthreads();
    }
    const int a = a0 + ty;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const int b = b0 + 4 * tx + e;
        if (a < j && b < j) part[((long long)blockIdx.x * j + a) * j + b] = acc[e];
    }
}

// G[a][b] = sum over chunks in order (a <= b), G[b][a] = conj(G[a][b]).
__global__ void k_gram_reduce(const double2 *__restrict__ part, int j, int nchunk, double2 *__restrict__ G) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < j * j; u += gridDim.x * blockDim.x) {
        const int a = u / j, b = u % j;
        if (a > b) continue;
        double2 s = make_double2(0.0, 0.0);
        for (int c = 0; c < nchunk; c++) {
            const double2 x = part[((long long)c * j + a) * j + b];
            s.x += x.x;
            s.y += x.y;
        }
        if (a == b) s.y = 0.0;
        G[a * j + b] = s;
        G[b * j + a] = make_double2(s.x, -s.y);
    }
}

// Jacobi eigen-decomposition of the Hermitian G (j x j, row-major), V <- V J
// accumulated on top of the identity.  On return G's diagonal holds the
// eigenvalues.  One block of 256 threads; *sweeps = sweeps taken.
__global__ void __launch_bounds__(256) k_jacobi(double2 *__restrict__ G, double2 *__restrict__ V, int j,
                                                int max_sweeps, int *sweeps) {
    __shared__ int sp[128], sq[128];
    __shared__ double sc[128], ss[128], sre[128], sim[128];
    __shared__ double red[2][8];
    __shared__ int s_stop;
    const int npad = j + (j & 1), np2 = npad / 2;
    for (int u = threadIdx.x; u < j * j; u += blockDim.x)
        V[u] = make_double2((u / j) == (u % j) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    int sw = 0;
    for (; sw < max_sweeps; sw++) {
        // convergence: off-diagonal Frobenius mass against the total
        double off = 0.0, tot = 0.0;
        for (int u = threadIdx.x; u < j * j; u += blockDim.x) {
            const double2 g = G[u];
            const double m2 = g.x * g.x + g.y * g.y;
            tot += m2;
            if ((u / j) != (u % j)) off += m2;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = off;
            red[1][threadIdx.x >> 5] = tot;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double o2 = 0.0, t2 = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
                o2 += red[0][w];
                t2 += red[1][w];
            }
            s_stop = !(o2 > 1e-30 * t2);
        }
        __syncthreads();
        if (s_stop) break;
        for (int step = 0; step < npad - 1; step++) {
            // round robin: position 0 fixed, the others rotate by one per step
            if (threadIdx.x < np2) {
                const int i = threadIdx.x;
                auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (npad - 1); };
                int p = at(i), q = at(npad - 1 - i);
                if (p > q) { int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0, pr = 1.0, pi = 0.0;
                if (q < j) {
                    const double2 g = G[p * j + q];
                    const double ag = sqrt(g.x * g.x + g.y * g.y);
                    const double a = G[p * j + p].x, b = G[q * j + q].x;
                    if (ag > 0.0 && ag > 1e-18 * sqrt(fabs(a * b))) {
                        const double tau = (b - a) / (2.0 * ag);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        pr = g.x / ag;
                        pi = g.y / ag;
                    }
                }
                sp[i] = p;
                sq[i] = q;
                sc[i] = c;
                ss[i] = s;
                sre[i] = pr;
                sim[i] = pi;
            }
            __syncthreads();
            // left: rows p, q of G <- J^H (rows)
            for (int u = threadIdx.x; u < np2 * j; u += blockDim.x) {
                const int i = u / j, r = u % j;
                const int p = sp[i], q = sq[i];
                if (q >= j || ss[i] == 0.0) continue;
                const double c = sc[i], s = ss[i];
                const double2 ph = make_double2(sre[i], sim[i]);
                const double2 gp = G[p * j + r], gq = G[q * j + r];
                const double2 e1 = cmul(ph, gq);                        // e^{i phi} G_qr
                const double2 e2 = cmulc(gp, ph);                       // e^{-i phi} G_pr
                G[p * j + r] = make_double2(c * gp.x - s * e1.x, c * gp.y - s * e1.y);
                G[q * j + r] = make_double2(s * e2.x + c * gq.x, s * e2.y + c * gq.y);
            }
            __syncthreads();
            // right: columns p, q of G and V <- (.) J
            for (int u = threadIdx.x; u < np2 * j; u += blockDim.x) {
                const int i = u / j, r = u % j;
                const int p = sp[i], q = sq[i];
                if (q >= j || ss[i] == 0.0) continue;
                const double c = sc[i], s = ss[i];
                const double2 ph = make_double2(sre[i], sim[i]);
#pragma unroll
                for (int w = 0; w < 2; w++) {
                    double2 *Mx = w ? V : G;
                    const double2 xp = Mx[r * j + p], xq = Mx[r * j + q];
                    const double2 f1 = cmulc(xq, ph);                   // e^{-i phi} x_q
                    const double2 f2 = cmul(ph, xp);                    // e^{i phi} x_p
                    Mx[r * j + p] = make_double2(c * xp.x - s * f1.x, c * xp.y - s * f1.y);
                    Mx[r * j + q] = make_double2(s * f2.x + c * xq.x, s * f2.y + c * xq.y);
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && sweeps) *sweeps = sw;
}

// B = W^H A for W (j x j) and A (j x M): B[a][m] = sum_l conj(W[l][a]) A[l][m].
__global__ void __launch_bounds__(256) k_transform(const double2 *__restrict__ W, const double2 *__restrict__ A,
                                                   long long ldA, int j, long long M, double2 *__restrict__ B,
                                                   long long ldB) {
    extern __shared__ double2 sw[];  // j x j
    for (int u = threadIdx.x; u < j * j; u += blockDim.x) sw[u] = W[u];
    __syncthreads();
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
        for (int a0 = 0; a0 < j; a0 += 8) {
            double2 acc[8];
#pragma unroll
            for (int e = 0; e < 8; e++) acc[e] = make_double2(0.0, 0.0);
            for (int l = 0; l < j; l++) {
                const double2 x = A[(long long)l * ldA + m];
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    if (a0 + e < j) {
                        const double2 w = sw[l * j + a0 + e];
                        acc[e].x = fma(w.x, x.x, fma(w.y, x.y, acc[e].x));
                        acc[e].y = fma(w.x, x.y, fma(-w.y, x.x, acc[e].y));
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 8; e++)
                if (a0 + e < j) B[(long long)(a0 + e) * ldB + m] = acc[e];
        }
    }
}

// After pass 2: V = V1 V2, eigenvalues lam = diag(G2); order by decreasing
// eigenvalue (ties: lower index first), sigma = sqrt(max(lam, 0)), and each
// column of V scaled so that its entry of largest magnitude (lowest row among
// equals) is real and positive.  One block.
__global__ void __launch_bounds__(256) k_recon_finish(const double2 *__restrict__ V1, const double2 *__restrict__ V2,
                                                      const double2 *__restrict__ G2, int j, double2 *__restrict__ Vout,
                                                      double *__restrict__ sigma, int *__restrict__ perm) {
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        const double li = G2[i * j + i].x;
        int rank = 0;
        for (int t = 0; t < j; t++) {
            const double lt = G2[t * j + t].x;
            rank += (lt > li) || (lt == li && t < i);
        }
        perm[rank] = i;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < j; c += blockDim.x) {
        const int src = perm[c];
        const double lam = G2[src * j + src].x;
        sigma[c] = sqrt(lam > 0.0 ? lam : 0.0);
        // column src of V1 V2, then its phase
        int pbest = 0;
        double abest = -1.0;
        for (int r = 0; r < j; r++) {
            double2 s = make_double2(0.0, 0.0);
            for (int l = 0; l < j; l++) {
                const double2 x = cmul(V1[r * j + l], V2[l * j + src]);
                s.x += x.x;
                s.y += x.y;
            }
            Vout[r * j + c] = s;
            const double a = sqrt(s.x * s.x + s.y * s.y);
            if (a > abest) {
                abest = a;
                pbest = r;
            }
        }
        const double2 vp = Vout[pbest * j + c];
        const double2 f = abest > 0.0 ? make_double2(vp.x / abest, -vp.y / abest) : make_double2(1.0, 0.0);
        for (int r = 0; r < j; r++) Vout[r * j + c] = cmul(Vout[r * j + c], f);
        Vout[pbest * j + c] = make_double2(abest, 0.0);
    }
}

// X[:, c] = sum_l Q[:, l] V[l][c], c < k (Q and X column-major).
__global__ void __launch_bounds__(256) k_recon_basis(const double2 *__restrict__ Q, long long ldQ, long long N, int j,
                                                     const double2 *__restrict__ V, int k, double2 *__restrict__ X,
                                                     long long ldX) {
    const int c = blockIdx.y;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int l = 0; l < j; l++) {
            const double2 x = cmul(Q[(long long)l * ldQ + i], V[l * j + c]);
            s.x += x.x;
            s.y += x.y;
        }
        X[(long long)c * ldX + i] = s;
    }
}

size_t recon_workspace(int j, long long M) {
    const long long nchunk = (M + kGramChunk - 1) / kGramChunk;
    return (size_t)nchunk * j * j * 16 + (size_t)j * M * 16 + (size_t)6 * j * j * 16 + (size_t)j * 4 + 4096;
}

// Pass 1 + pass 2 on C; sigma and the phase-normalised V land in sigma / V.
cudaError_t launch_recon_svd(const double2 *C, long long ldC, int j, long long M, void *ws, double *sigma,
                             double2 *V, int *sweeps, cudaStream_t s) {
    const long long chunk = kGramChunk;
    const int nchunk = (int)((M + chunk - 1) / chunk);
    char *w = (char *)ws;
    double2 *part = (double2 *)w;
    w += (size_t)nchunk * j * j * 16;
    double2 *B = (double2 *)w;
    w += (size_t)j * M * 16;
    double2 *G1 = (double2 *)w, *V1 = G1 + j * j, *G2 = V1 + j * j, *V2 = G2 + j * j;
    w += (size_t)6 * j * j * 16;
    int *perm = (int *)w;
    const int nt = (j + RT - 1) / RT;
    dim3 gg(nchunk, nt, nt);
    const int gr = (j * j + 255) / 256;
    k_gram_part<<<gg, 256, 0, s>>>(C, ldC, j, M, chunk, part);
    k_gram_reduce<<<gr, 256, 0, s>>>(part, j, nchunk, G1);
    k_jacobi<<<1, 256, 0, s>>>(G1, V1, j, 40, sweeps);
    const size_t tsm = (size_t)j * j * 16;
    if (tsm > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_transform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm);
        if (e != cudaSuccess) return e;
    }
    long long gt = (M + 255) / 256;
    if (gt > 152 * 4) gt = 152 * 4;
    k_transform<<<(int)gt, 256, tsm, s>>>(V1, C, ldC, j, M, B, M);
    k_gram_part<<<gg, 256, 0, s>>>(B, M, j, M, chunk, part);
    k_gram_reduce<<<gr, 256, 0, s>>>(part, j, nchunk, G2);
    k_jacobi<<<1, 256, 0, s>>>(G2, V2, j, 40, sweeps ? sweeps + 1 : nullptr);
    k_recon_finish<<<1, 256, 0, s>>>(V1, V2, G2, j, V, sigma, perm);
    return cudaGetLastError();
}

cudaError_t launch_recon_basis(const double2 *Q, long long ldQ, long long N, int j, const double2 *V, int k,
                               double2 *X, long long ldX, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    long long g = (N + 255) / 256;
    if (g > 1024) g = 1024;
    k_recon_basis<<<dim3((unsigned)g, (unsigned)k), 256, 0, s>>>(Q, ldQ, N, j, V, k, X, ldX);
    return cudaGetLastError();
}

}  // namespace rbk
