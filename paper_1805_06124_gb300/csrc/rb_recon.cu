// rb_recon.cu -- the reconstruction step (Alg. 4, Sec. 5.2.2): the singular
// value decomposition of R(1:j, 1:M) = C = Q_j^H S and the enriched basis
// X_k = Q_j V(:, 1:k).
//
// Only the left factor of C (j x M, j small, M large) is needed, so the SVD is
// taken through j x j Gram matrices, in two passes:
//   pass 1  G1 = C C^H in FP32, Jacobi in FP32 -> V1, then made unitary to
//           FP64 precision by Newton-Schulz steps V <- V (3I - V^H V) / 2;
//   pass 2  B = V1^H C and G2 = B B^H in double-float (FP32 pairs, about 48
//           bits, every product relative to its own operands), Jacobi in FP64
//           on G2 with V accumulated on top of V1 -> V = V1 V2, lambda = diag.
// G2 is nearly diagonal with off-diagonal entries small relative to
// sqrt(G2_aa G2_bb), so pass 2 takes two or three sweeps and, with the
// relative rotation threshold below, keeps the small singular values to high
// relative accuracy (the squaring in a one-pass Gram method would lose them).
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, so
// everything of size O(j^2 M) is FP32 or double-float; FP64 is left to the
// j x j work.
//
// Jacobi: cyclic, parallel ("round robin") ordering -- every step rotates
// npad/2 disjoint index pairs at once: left updates of all pairs, a barrier,
// right updates, a barrier; G (and V where it fits) in shared memory, one
// block.  For a pair (p, q) with g = G_pq = |g| e^{i phi}: tau = (G_qq -
// G_pp) / (2|g|), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 +
// t^2), s = t c, J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] on columns (p, q);
// G <- J^H G J, V <- V J.  A pair is rotated only while |g| > eps
// sqrt(|G_pp G_qq|) (the relative criterion of Demmel and Veselic); a sweep
// with no rotation ends the iteration.
//
// C is scaled by a power of two 2^-E (max |c| < 1) before any FP32 work so
// that no square over- or underflows for representable inputs; sigma is
// scaled back.  All sums run in a fixed order: results are deterministic.
#include "rb_internal.cuh"

namespace rbk {

constexpr int RG_T = 32;          // columns per staged tile
constexpr int RG_THREADS = 512;   // Gram block (triangle of entries)
constexpr int RG_MAXE = 13;       // entries per thread: ceil(112 * 113 / 2 / 512)
constexpr int RG_MAXE_S = 4;      // the same for j <= 63 (2016 entries)
constexpr int RJ_THREADS = 512;   // Jacobi block
constexpr int RJ_PAIRS = 64;      // index pairs per step (j <= 128)
constexpr int RT_THREADS = 256;   // transform block
constexpr int RT_ROWS = 14;       // output rows per warp: ceil(112 / 8)
constexpr int RT_ROWS_S = 7;      // the same for j <= 56
constexpr int kMaxJ = 112;
constexpr int kJacobiMaxSweeps = 60;

// Largest biased exponent over C (integer max on the IEEE bits).
__global__ void k_max_exp(const double2 *__restrict__ A, long long ldA, int j, long long M, int *__restrict__ emax) {
    unsigned int e = 0;
    for (int r = blockIdx.y; r < j; r += gridDim.y)
        for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
            const double2 v = A[(long long)r * ldA + m];
            e = max(e, max((unsigned int)(__double_as_longlong(v.x) >> 52) & 0x7FFu,
                           (unsigned int)(__double_as_longlong(v.y) >> 52) & 0x7FFu));
        }
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0 && e) atomicMax(emax, (int)e);
}

// 2^-E with E = e_max - 1022 (max |c| < 2^E); 1 for an all-zero C.
__device__ __forceinline__ double c_scale(const int *emax) {
    const int e = *emax;
    return e ? ldexp(1.0, 1022 - e) : 1.0;
}

__device__ __forceinline__ float4 split_c(double2 v) {
    float4 r;
    split_rn(v.x, r.x, r.z);
    split_rn(v.y, r.y, r.w);
    return r;  // (re hi, im hi, re lo, im lo)
}

// Partial Gram sums over one column chunk: part[(chunk * j + a) * j + b] =
// sum_{m in chunk} A[a][m] conj(A[b][m]) (times the scale^2) for a <= b.
// The block stages RG_T columns of all j rows in shared memory; thread t
// owns the upper-triangle entries e = t + RG_THREADS i (row-major order).
// DF: double-float products and sums; otherwise FP32.
template <bool DF, int MAXE>
__global__ void __launch_bounds__(RG_THREADS, MAXE <= RG_MAXE_S ? 2 : 1) k_gram_tri(const double2 *__restrict__ A, long long ldA, int j,
                                                          long long M, long long chunk, const int *__restrict__ emax,
                                                          double2 *__restrict__ part) {
    extern __shared__ float4 st[];  // j x (RG_T + 1)
    const int ne = j * (j + 1) / 2;
    const double sc = emax ? c_scale(emax) : 1.0;
    int eab[MAXE];  // row offsets of a (low 16 bits) and b (high 16 bits) in the tile
    float acc[MAXE][4];
#pragma unroll
    for (int i = 0; i < MAXE; i++) {
        int e = threadIdx.x + RG_THREADS * i, a = 0;
        while (a < j && e >= j - a) {
            e -= j - a;
            a++;
        }
        eab[i] = a < j ? (a * (RG_T + 1)) | ((a + e) * (RG_T + 1)) << 16 : 0;
        acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    }
    const long long m0 = (long long)blockIdx.x * chunk, m1 = m0 + chunk < M ? m0 + chunk : M;
    for (long long mt = m0; mt < m1; mt += RG_T) {
        __syncthreads();
        for (int u = threadIdx.x; u < j * RG_T; u += RG_THREADS) {
            const int r = u / RG_T, c = u % RG_T;
            const long long m = mt + c;
            double2 v = m < m1 ? A[(long long)r * ldA + m] : make_double2(0.0, 0.0);
            v.x *= sc;
            v.y *= sc;
            st[r * (RG_T + 1) + c] =
                DF ? split_c(v) : make_float4(__double2float_rn(v.x), __double2float_rn(v.y), 0.f, 0.f);
        }
        __syncthreads();
        const int nc = m1 - mt < RG_T ? (int)(m1 - mt) : RG_T;
        for (int c = 0; c < nc; c++) {
#pragma unroll
            for (int i = 0; i < MAXE; i++) {
                if (RG_THREADS * i >= ne) break;
                if ((int)threadIdx.x + RG_THREADS * i < ne) {
                    const float4 x = st[(eab[i] & 0xFFFF) + c], y = st[(eab[i] >> 16) + c];
                    if (DF) {
                        // x conj(y) = conj(y) x
                        df_cmac(acc[i][0], acc[i][1], acc[i][2], acc[i][3], y.x, y.y, y.z, y.w, x.x, x.y, x.z, x.w);
                    } else {
                        acc[i][0] = fmaf(x.x, y.x, fmaf(x.y, y.y, acc[i][0]));
                        acc[i][2] = fmaf(x.y, y.x, fmaf(-x.x, y.y, acc[i][2]));
                    }
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < MAXE; i++) {
        if ((int)threadIdx.x + RG_THREADS * i < ne)
            part[((long long)blockIdx.x * j + (eab[i] & 0xFFFF) / (RG_T + 1)) * j + (eab[i] >> 16) / (RG_T + 1)] =
                make_double2((double)acc[i][0] + (double)acc[i][1], (double)acc[i][2] + (double)acc[i][3]);
    }
}

// G[a][b] = sum over the chunks' partial sums (a <= b), G[b][a] =
// conj(G[a][b]).  One warp per entry: lane l adds chunks l, l + 32, ... in
// order, then a fixed butterfly combines the lanes (deterministic).
__global__ void k_gram_reduce(const double2 *__restrict__ part, int j, int nchunk, double2 *__restrict__ G) {
    const int ne = j * (j + 1) / 2, lane = threadIdx.x & 31;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ne; w += (gridDim.x * blockDim.x) >> 5) {
        int e = w, a = 0;
        while (e >= j - a) {
            e -= j - a;
            a++;
        }
        const int b = a + e;
        double sx = 0.0, sy = 0.0;
        for (int c = lane; c < nchunk; c += 32) {
            const double2 x = part[((long long)c * j + a) * j + b];
            sx += x.x;
            sy += x.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) {
            if (a == b) sy = 0.0;
            G[a * j + b] = make_double2(sx, sy);
            G[b * j + a] = make_double2(sx, -sy);
        }
    }
}

// ------------------------------------------------------------------ Jacobi
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename T> __device__ __forceinline__ T cx(double re, double im);
template <> __device__ __forceinline__ float2 cx<float2>(double re, double im) {
    return make_float2((float)re, (float)im);
}
template <> __device__ __forceinline__ double2 cx<double2>(double re, double im) { return make_double2(re, im); }

template <typename T> __device__ __forceinline__ T cmul_t(T a, T b) {  // a b
    T r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename T> __device__ __forceinline__ T cmulc_t(T a, T b) {  // a conj(b)
    T r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}

// Hermitian Jacobi on G (j x j, FP64 input, row-major) in precision R, G in
// shared memory, one block.  A step rotates the npad/2 disjoint pairs of the
// round-robin ordering at once; G <- J^H G J is formed block by block over the
// upper triangle of 2 x 2 pair blocks (rows of pair i, columns of pair i2,
// i <= i2: the left rotation of i, then the right rotation of i2, the mirror
// entries by Hermitian symmetry), the diagonal blocks in closed form (G_pp -=
// t|g|, G_qq += t|g|, G_pq = 0).  Every entry belongs to one block, so a step
// needs one barrier after the rotation parameters and one after the update.
// The rotations are recorded (c, s, phase) in rec, step by step, for
// k_apply_rot; V is not formed here.  The eigenvalues (diag of the rotated G)
// go to lam; stats gets the sweeps that rotated and the rotations applied.
constexpr int RJ_BLK = 4;  // pair blocks per thread: ceil(56 * 57 / 2 / 512)

struct __align__(32) Rot {  // one recorded rotation: c, s, e^{i phi}
    double c, s, px, py;
};

template <typename R>
__global__ void __launch_bounds__(RJ_THREADS) k_jacobi(const double2 *__restrict__ Gin, int j, double eps, int max_sweeps,
                                                       double *__restrict__ lam, int *__restrict__ stats,
                                                       Rot *__restrict__ rec) {
    using T = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char jsm[];
    T *G = reinterpret_cast<T *>(jsm);
    __shared__ int sp[RJ_PAIRS], sq[RJ_PAIRS];
    __shared__ R sc[RJ_PAIRS], ss[RJ_PAIRS], stg[RJ_PAIRS];  // c, s, t |g|
    __shared__ T sph[RJ_PAIRS];
    __shared__ int s_rot;
    const int npad = j + (j & 1), np2 = npad / 2, nblk = np2 * (np2 + 1) / 2;
    for (int u = threadIdx.x; u < j * j; u += blockDim.x) {
        const double2 g = Gin[u];
        G[u] = cx<T>(g.x, g.y);
    }
    int blk[RJ_BLK];  // (i, i2) with i <= i2, packed i | i2 << 8
#pragma unroll
    for (int b = 0; b < RJ_BLK; b++) {
        int u = threadIdx.x + b * RJ_THREADS, i = 0;
        while (i < np2 && u >= np2 - i) {
            u -= np2 - i;
            i++;
        }
        blk[b] = i < np2 ? (i | (i + u) << 8) : 0;
    }
    __syncthreads();
    const R e = (R)eps;
    const T zero = cx<T>(0.0, 0.0);
    int sw = 0, nrot = 0;
    for (; sw < max_sweeps; sw++) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        for (int step = 0; step < npad - 1; step++) {
            // round robin: position 0 fixed, the others rotate by one per step
            if ((int)threadIdx.x < np2) {
                const int i = threadIdx.x;
                auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (npad - 1); };
                int p = at(i), q = at(npad - 1 - i);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                R c = 1, s = 0, tg = 0;
                T ph = cx<T>(1.0, 0.0);
                if (q < j) {
                    // few square roots and divisions: they are long sequences
                    // on this GPU's FP64 pipe
                    const T g = G[p * j + q];
                    const R g2 = g.x * g.x + g.y * g.y;
                    const R a = G[p * j + p].x, b = G[q * j + q].x;
                    if (g2 > (R)0 && g2 > e * e * fabs(a * b)) {
                        const R rg = rsqrt(g2), ag = g2 * rg;  // 1/|g|, |g|
                        const R tau = (b - a) * (R)0.5 * rg;
                        const R at_ = fabs(tau);
                        R t = at_ > (R)1e15 ? (R)0.5 / at_ : (R)1 / (at_ + sqrt((R)1 + tau * tau));
                        if (tau < (R)0) t = -t;
                        c = rsqrt((R)1 + t * t);
                        s = t * c;
                        tg = t * ag;
                        ph.x = g.x * rg;
                        ph.y = g.y * rg;
                        if (s != (R)0) atomicAdd(&s_rot, 1);
                    }
                }
                sp[i] = p;
                sq[i] = q;
                sc[i] = c;
                ss[i] = s;
                stg[i] = tg;
                sph[i] = ph;
                if (sw < max_sweeps)
                    rec[((long long)sw * (npad - 1) + step) * RJ_PAIRS + i] =
                        Rot{(double)c, (double)s, (double)ph.x, (double)ph.y};
            }
            __syncthreads();
#pragma unroll
            for (int bb = 0; bb < RJ_BLK; bb++) {
                if ((int)threadIdx.x + bb * RJ_THREADS >= nblk) break;
                const int i = blk[bb] & 0xFF, i2 = blk[bb] >> 8;
                const R s1 = ss[i], s2 = ss[i2];
                if (s1 == (R)0 && s2 == (R)0) continue;
                const int p = sp[i], q = sq[i];
                if (i == i2) {  // rotated pair: closed form
                    const R tg = stg[i];
                    T gp = G[p * j + p], gq = G[q * j + q];
                    gp.x -= tg;
                    gp.y = 0;
                    gq.x += tg;
                    gq.y = 0;
                    G[p * j + p] = gp;
                    G[q * j + q] = gq;
                    G[p * j + q] = zero;
                    G[q * j + p] = zero;
                    continue;
                }
                const int p2 = sp[i2], q2 = sq[i2];
                const bool vq = q < j, vq2 = q2 < j;
                T x00 = G[p * j + p2], x01 = vq2 ? G[p * j + q2] : zero, x10 = vq ? G[q * j + p2] : zero,
                  x11 = (vq && vq2) ? G[q * j + q2] : zero;
                if (s1 != (R)0) {  // rows (p, q) <- J_i^H
                    const R c = sc[i];
                    const T ph = sph[i];
                    const T a0 = cmul_t(ph, x10), a1 = cmul_t(ph, x11);      // e^{i phi} x_q.
                    const T b0 = cmulc_t(x00, ph), b1 = cmulc_t(x01, ph);    // e^{-i phi} x_p.
                    T n00, n01, n10, n11;
                    n00.x = c * x00.x - s1 * a0.x; n00.y = c * x00.y - s1 * a0.y;
                    n01.x = c * x01.x - s1 * a1.x; n01.y = c * x01.y - s1 * a1.y;
                    n10.x = s1 * b0.x + c * x10.x; n10.y = s1 * b0.y + c * x10.y;
                    n11.x = s1 * b1.x + c * x11.x; n11.y = s1 * b1.y + c * x11.y;
                    x00 = n00; x01 = n01; x10 = n10; x11 = n11;
                }
                if (s2 != (R)0) {  // columns (p2, q2) <- (.) J_i2
                    const R c = sc[i2];
                    const T ph = sph[i2];
                    const T f0 = cmulc_t(x01, ph), f1 = cmulc_t(x11, ph);    // e^{-i phi} x_.q
                    const T h0 = cmul_t(ph, x00), h1 = cmul_t(ph, x10);      // e^{i phi} x_.p
                    T n00, n01, n10, n11;
                    n00.x = c * x00.x - s2 * f0.x; n00.y = c * x00.y - s2 * f0.y;
                    n10.x = c * x10.x - s2 * f1.x; n10.y = c * x10.y - s2 * f1.y;
                    n01.x = s2 * h0.x + c * x01.x; n01.y = s2 * h0.y + c * x01.y;
                    n11.x = s2 * h1.x + c * x11.x; n11.y = s2 * h1.y + c * x11.y;
                    x00 = n00; x01 = n01; x10 = n10; x11 = n11;
                }
                auto put = [&](int r, int cc, T v) {
                    G[r * j + cc] = v;
                    v.y = -v.y;
                    G[cc * j + r] = v;
                };
                put(p, p2, x00);
                if (vq2) put(p, q2, x01);
                if (vq) put(q, p2, x10);
                if (vq && vq2) put(q, q2, x11);
            }
            __syncthreads();
        }
        const int any = s_rot;
        nrot += any;
        __syncthreads();
        if (!any) break;
    }
    for (int a = threadIdx.x; a < j; a += blockDim.x) lam[a] = (double)G[a * j + a].x;
    if (threadIdx.x == 0 && stats) {
        stats[0] = sw;    // sweeps with at least one rotation (all recorded)
        stats[1] = nrot;  // rotations applied
    }
}

// V <- Vinit (identity when null) times the recorded rotations of the first
// stats[0] sweeps, in order.  Rows of V are independent under V <- V J: block
// r keeps row r in shared memory and thread i applies pair i of each step
// (the same round-robin pairs), one barrier per step; the records come in
// batches of RA_BATCH steps, copied to shared memory with coalesced loads.
// FP64 arithmetic on the recorded values (FP32 rotations of pass 1 are unitary
// only to FP32 precision; the Newton-Schulz steps that follow fix that).
constexpr int RA_BATCH = 16;

__global__ void __launch_bounds__(128) k_apply_rot(const Rot *__restrict__ rec, const int *__restrict__ stats, int j,
                                                   const double2 *__restrict__ Vinit, double2 *__restrict__ Vout) {
    __shared__ double2 row[128];
    __shared__ Rot srec[RA_BATCH * RJ_PAIRS];
    const int r = blockIdx.x;
    const int npad = j + (j & 1), np2 = npad / 2;
    for (int c = threadIdx.x; c < j; c += blockDim.x)
        row[c] = Vinit ? Vinit[r * j + c] : make_double2(c == r ? 1.0 : 0.0, 0.0);
    const long long nsteps = (long long)stats[0] * (npad - 1);
    for (long long t0 = 0; t0 < nsteps; t0 += RA_BATCH) {
        const int nb = nsteps - t0 < RA_BATCH ? (int)(nsteps - t0) : RA_BATCH;
        __syncthreads();
        for (int u = threadIdx.x; u < nb * RJ_PAIRS; u += blockDim.x) srec[u] = rec[t0 * RJ_PAIRS + u];
        __syncthreads();
        for (int b = 0; b < nb; b++) {
            const long long t = t0 + b;
            const int step = (int)(t % (npad - 1)), i = threadIdx.x;
            if (i < np2) {
                auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (npad - 1); };
                int p = at(i), q = at(npad - 1 - i);
                if (p > q) {
                    const int tt = p;
                    p = q;
                    q = tt;
                }
                const Rot g = srec[b * RJ_PAIRS + i];
                if (q < j && g.s != 0.0) {
                    const double c = g.c, s = g.s;
                    const double2 ph = make_double2(g.px, g.py);
                    const double2 xp = row[p], xq = row[q];
                    const double2 f1 = cmulc_t(xq, ph), f2 = cmul_t(ph, xp);
                    row[p] = make_double2(c * xp.x - s * f1.x, c * xp.y - s * f1.y);
                    row[q] = make_double2(s * f2.x + c * xq.x, s * f2.y + c * xq.y);
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < j; c += blockDim.x) Vout[r * j + c] = row[c];
}

// ----------------------------------------------------- Newton-Schulz step
// E = V^H V: E[r][c] = sum_l conj(V[l][r]) V[l][c].  Block r, thread c.
__global__ void k_vhv(const double2 *__restrict__ V, int j, double2 *__restrict__ E) {
    const int r = blockIdx.x, c = threadIdx.x;
    if (c >= j) return;
    double sx = 0.0, sy = 0.0;
    for (int l = 0; l < j; l++) {
        const double2 a = V[l * j + r], b = V[l * j + c];
        sx = fma(a.x, b.x, fma(a.y, b.y, sx));
        sy = fma(a.x, b.y, fma(-a.y, b.x, sy));
    }
    E[r * j + c] = make_double2(sx, sy);
}

// Vn = V (3I - E) / 2: Vn[r][c] = 1.5 V[r][c] - 0.5 sum_l V[r][l] E[l][c].
// With Vs != nullptr the result is also written split into FP32 pairs.
__global__ void k_ns_update(const double2 *__restrict__ V, const double2 *__restrict__ E, int j,
                            double2 *__restrict__ Vn, float4 *__restrict__ Vs) {
    const int r = blockIdx.x, c = threadIdx.x;
    if (c >= j) return;
    double sx = 0.0, sy = 0.0;
    for (int l = 0; l < j; l++) {
        const double2 a = V[r * j + l], b = E[l * j + c];
        sx = fma(a.x, b.x, fma(-a.y, b.y, sx));
        sy = fma(a.x, b.y, fma(a.y, b.x, sy));
    }
    const double2 v = V[r * j + c];
    const double2 o = make_double2(1.5 * v.x - 0.5 * sx, 1.5 * v.y - 0.5 * sy);
    Vn[r * j + c] = o;
    if (Vs) Vs[r * j + c] = split_c(o);
}

// ------------------------------------------------------------- transform
// B[a][m] = sum_l conj(V[l][a]) C[l][m] (times the scale) in double-float.
// Lane = column within a tile of 32, warp w = rows a = w + 8 i.  The C tile
// (j x 32, split) sits in shared memory; V (split) is read with warp-wide
// broadcast loads.
template <int ROWS>
__global__ void __launch_bounds__(RT_THREADS, ROWS <= RT_ROWS_S ? 3 : 1) k_transform_df(const float4 *__restrict__ Vsp, const double2 *__restrict__ C,
                                                             long long ldC, int j, long long M,
                                                             const int *__restrict__ emax, double2 *__restrict__ B,
                                                             long long ldB) {
    extern __shared__ float4 tsm[];  // j x 32
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double sc = c_scale(emax);
    for (long long mt = (long long)blockIdx.x * 32; mt < M; mt += (long long)gridDim.x * 32) {
        __syncthreads();
        for (int u = threadIdx.x; u < j * 32; u += RT_THREADS) {
            const int r = u >> 5, c = u & 31;
            const long long m = mt + c;
            double2 v = m < M ? C[(long long)r * ldC + m] : make_double2(0.0, 0.0);
            v.x *= sc;
            v.y *= sc;
            tsm[u] = split_c(v);
        }
        __syncthreads();
        float acc[ROWS][4];
#pragma unroll
        for (int i = 0; i < ROWS; i++) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
        for (int l = 0; l < j; l++) {
            const float4 x = tsm[l * 32 + lane];
#pragma unroll
            for (int i = 0; i < ROWS; i++) {
                const int a = w + 8 * i;
                if (a < j) {
                    const float4 v = __ldg(Vsp + l * j + a);
                    df_cmac(acc[i][0], acc[i][1], acc[i][2], acc[i][3], v.x, v.y, v.z, v.w, x.x, x.y, x.z, x.w);
                }
            }
        }
        const long long m = mt + lane;
        if (m < M) {
#pragma unroll
            for (int i = 0; i < ROWS; i++) {
                const int a = w + 8 * i;
                if (a < j)
                    B[(long long)a * ldB + m] =
                        make_double2((double)acc[i][0] + (double)acc[i][1], (double)acc[i][2] + (double)acc[i][3]);
            }
        }
    }
}

// ---------------------------------------------------------------- finish
// Order by decreasing eigenvalue (ties: lower index first), sigma =
// sqrt(max(lam, 0)) 2^E, and each column of V scaled so that its entry of
// largest magnitude (lowest row among equals) is real and positive.
__global__ void __launch_bounds__(256) k_recon_finish(const double *__restrict__ lam, const double2 *__restrict__ Vin,
                                                      int j, const int *__restrict__ emax, double2 *__restrict__ Vout,
                                                      double *__restrict__ sigma, int *__restrict__ perm) {
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        const double li = lam[i];
        int rank = 0;
        for (int t = 0; t < j; t++) {
            const double lt = lam[t];
            rank += (lt > li) || (lt == li && t < i);
        }
        perm[rank] = i;
    }
    __syncthreads();
    const double unscale = 1.0 / c_scale(emax);  // 2^E, exact
    for (int c = threadIdx.x; c < j; c += blockDim.x) {
        const int src = perm[c];
        const double l = lam[src];
        sigma[c] = sqrt(l > 0.0 ? l : 0.0) * unscale;
        int pbest = 0;
        double abest = -1.0;
        for (int r = 0; r < j; r++) {
            const double2 v = Vin[r * j + src];
            const double a = sqrt(v.x * v.x + v.y * v.y);
            if (a > abest) {
                abest = a;
                pbest = r;
            }
        }
        const double2 vp = Vin[pbest * j + src];
        const double2 f = abest > 0.0 ? make_double2(vp.x / abest, -vp.y / abest) : make_double2(1.0, 0.0);
        for (int r = 0; r < j; r++) Vout[r * j + c] = cmul_t(Vin[r * j + src], f);
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
            const double2 x = cmul_t(Q[(long long)l * ldQ + i], V[l * j + c]);
            s.x += x.x;
            s.y += x.y;
        }
        X[(long long)c * ldX + i] = s;
    }
}

// ---------------------------------------------------------------- host side
namespace {
int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
        n = 148;
    return n;
}
long long gram_chunk(long long M, int nsm) {
    const long long nchunk = 2LL * nsm;
    long long ch = (M + nchunk - 1) / nchunk;
    ch = (ch + RG_T - 1) / RG_T * RG_T;
    return ch < RG_T ? RG_T : ch;
}
size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

struct ReconWs {
    int *emax, *stats;
    double2 *part, *B, *G1, *G2, *Va, *Vb, *E;
    float4 *Vsp;
    Rot *rec;
    double *lam;
    int *perm;
    size_t total;
};
ReconWs carve(void *base, int j, long long M, int nsm) {
    const long long chunk = gram_chunk(M, nsm);
    const long long nchunk = (M + chunk - 1) / chunk;
    const size_t jj = (size_t)j * j;
    ReconWs w;
    char *p = (char *)base;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *r = p ? p + off : nullptr;
        off += up256(bytes);
        return r;
    };
    w.emax = (int *)take(16);
    w.stats = (int *)take(16);
    w.part = (double2 *)take((size_t)nchunk * jj * 16);
    w.B = (double2 *)take((size_t)j * M * 16);
    w.G1 = (double2 *)take(jj * 16);
    w.G2 = (double2 *)take(jj * 16);
    w.Va = (double2 *)take(jj * 16);
    w.Vb = (double2 *)take(jj * 16);
    w.E = (double2 *)take(jj * 16);
    w.Vsp = (float4 *)take(jj * 16);
    w.lam = (double *)take((size_t)j * 8);
    w.perm = (int *)take((size_t)j * 4);
    w.rec = (Rot *)take((size_t)kJacobiMaxSweeps * (j + 1) * RJ_PAIRS * 32);
    w.total = off;
    return w;
}

template <typename R> size_t jacobi_smem(int j) { return (size_t)j * j * sizeof(typename Cx<R>::T); }

template <typename R>
cudaError_t launch_jacobi(const double2 *G, int j, double eps, double *lam, int *stats, Rot *rec, cudaStream_t s) {
    const size_t sm = jacobi_smem<R>(j);
    cudaError_t e = cudaFuncSetAttribute(k_jacobi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_jacobi<R><<<1, RJ_THREADS, sm, s>>>(G, j, eps, kJacobiMaxSweeps, lam, stats, rec);
    return cudaGetLastError();
}
}  // namespace

size_t recon_workspace(int j, long long M) { return carve(nullptr, j, M, sm_count()).total; }

// Pass 1 + pass 2 on C; sigma and the phase-normalised V land in sigma / V.
// stats (optional, device, 4 ints): sweeps and rotations of the pass-1 and
// pass-2 Jacobi iterations.  ev (optional, 7 events) is recorded at the start
// and after each phase: pass-1 Gram, pass-1 Jacobi, Newton-Schulz, transform,
// pass-2 Gram, pass-2 Jacobi + ordering.
cudaError_t launch_recon_svd(const double2 *C, long long ldC, int j, long long M, void *ws, double *sigma,
                             double2 *V, int *stats, cudaEvent_t *ev, cudaStream_t s) {
    if (j < 1 || j > kMaxJ) return cudaErrorInvalidValue;
    const int nsm = sm_count();
    const ReconWs w = carve(ws, j, M, nsm);
    const long long chunk = gram_chunk(M, nsm);
    const int nchunk = (int)((M + chunk - 1) / chunk);
    const int gr = (j * (j + 1) / 2 + 7) / 8;  // one warp per entry, 8 warps per block
    const size_t gsm = (size_t)j * (RG_T + 1) * 16;
    cudaError_t e;
    // register arrays sized for the largest j, or for j <= 63 / 56 (more
    // warps per SM on the common sizes)
    const bool small = j <= 56;
    auto gram32 = small ? k_gram_tri<false, RG_MAXE_S> : k_gram_tri<false, RG_MAXE>;
    auto gramdf = small ? k_gram_tri<true, RG_MAXE_S> : k_gram_tri<true, RG_MAXE>;
    auto transf = small ? k_transform_df<RT_ROWS_S> : k_transform_df<RT_ROWS>;
    if ((e = cudaFuncSetAttribute(gram32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(gramdf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm)) != cudaSuccess)
        return e;
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    if ((e = mark(0)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.emax, 0, 16, s)) != cudaSuccess) return e;
    long long gx = (M + 255) / 256;
    if (gx > 2LL * nsm) gx = 2LL * nsm;
    k_max_exp<<<dim3((unsigned)gx, (unsigned)(j < 8 ? j : 8)), 256, 0, s>>>(C, ldC, j, M, w.emax);
    // pass 1: FP32 Gram and Jacobi
    gram32<<<nchunk, RG_THREADS, gsm, s>>>(C, ldC, j, M, chunk, w.emax, w.part);
    k_gram_reduce<<<gr, 256, 0, s>>>(w.part, j, nchunk, w.G1);
    if ((e = mark(1)) != cudaSuccess) return e;
    if ((e = launch_jacobi<float>(w.G1, j, 0x1p-22, w.lam, w.stats, w.rec, s)) != cudaSuccess) return e;
    k_apply_rot<<<j, 128, 0, s>>>(w.rec, w.stats, j, nullptr, w.Va);
    if ((e = mark(2)) != cudaSuccess) return e;
    // V1 unitary to FP64 precision: three Newton-Schulz steps (the FP32
    // rotations leave ||V^H V - I|| near 1e-5; each step squares it)
    double2 *cur = w.Va, *nxt = w.Vb;
    const int nt = (j + 31) / 32 * 32;
    for (int it = 0; it < 3; it++) {
        k_vhv<<<j, nt, 0, s>>>(cur, j, w.E);
        k_ns_update<<<j, nt, 0, s>>>(cur, w.E, j, nxt, it == 2 ? w.Vsp : nullptr);
        double2 *t = cur;
        cur = nxt;
        nxt = t;
    }
    if ((e = mark(3)) != cudaSuccess) return e;
    // pass 2: B = V1^H C, G2 = B B^H in double-float, Jacobi in FP64 from V1
    const size_t tsm = (size_t)j * 32 * 16;
    if ((e = cudaFuncSetAttribute(transf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm)) != cudaSuccess)
        return e;
    long long gt = (M + 31) / 32;
    if (gt > 6LL * nsm) gt = 6LL * nsm;
    transf<<<(unsigned)gt, RT_THREADS, tsm, s>>>(w.Vsp, C, ldC, j, M, w.emax, w.B, M);
    if ((e = mark(4)) != cudaSuccess) return e;
    gramdf<<<nchunk, RG_THREADS, gsm, s>>>(w.B, M, j, M, chunk, nullptr, w.part);
    k_gram_reduce<<<gr, 256, 0, s>>>(w.part, j, nchunk, w.G2);
    if ((e = mark(5)) != cudaSuccess) return e;
    if ((e = launch_jacobi<double>(w.G2, j, 0x1p-52, w.lam, w.stats + 2, w.rec, s)) != cudaSuccess) return e;
    k_apply_rot<<<j, 128, 0, s>>>(w.rec, w.stats + 2, j, cur, nxt);
    k_recon_finish<<<1, 256, 0, s>>>(w.lam, nxt, j, w.emax, V, sigma, w.perm);
    if (stats && (e = cudaMemcpyAsync(stats, w.stats, 4 * sizeof(int), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return mark(6);
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
