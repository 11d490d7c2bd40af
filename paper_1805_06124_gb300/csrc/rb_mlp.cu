// rb_mlp.cu -- the learned surrogate: an MLP (q, m) -> 2k real outputs
// (Re/Im of a snapshot's basis coefficients c = Q^H s), widths
// 2 -> 256 -> 256 -> 256 -> 2k, exact-erf GELU, BF16 weights with FP32 master
// copies, FP32 accumulation, Adam with cosine learning-rate decay.
//
// The three 256-wide layers and all their backward products run on the
// fifth-generation tensor cores (tcgen05, BF16 x BF16 -> FP32 in TMEM) with
// fused epilogues; the 2-input first layer and the reductions run on CUDA
// cores.  One training step is captured in a CUDA graph and replayed; the
// step counter, batch offset and learning rate live on the device.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "rb_internal.cuh"
#include "rb_tc.cuh"

typedef __nv_bfloat16 bf16;

namespace rbk {

constexpr int MW = 256;    // hidden width
constexpr int GT = 128;    // GEMM tile (M and N)
constexpr int GKC = 64;    // K per stage

enum { EPI_STORE = 0, EPI_BIAS_GELU = 1, EPI_GELU_BWD = 2 };

struct GemmArgs {
    int M, N, K;
    const bf16 *A;
    long long sam, sak;  // A(m, k) = A[m*sam + k*sak]
    const bf16 *B;
    long long sbn, sbk;  // B(n, k) = B[n*sbn + k*sbk]
    int epi;
    const float *bias;   // [N] or null
    float *out;          // FP32 (m, n) at out[m*ldo + n]
    long long ldo;
    bf16 *outb;          // BF16 copy (m, n) at outb[m*ldb + n] or null
    long long ldb;
    const float *zin;    // pre-activation for EPI_GELU_BWD, (m, n) at zin[m*ldz + n]
    long long ldz;
    float *outh;         // FP32 gelu(z) (EPI_BIAS_GELU) at outh[m*ldo + n], or null
    const float *Af;     // split form: FP32 A and B (same strides as A, B)
    const float *Bf;
    int *err;
    unsigned long long wait;  // budget of each mbarrier wait, SM clock cycles
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Stage rows [r0, r0+GT) x k [k0, k0+KC) of a strided BF16 matrix into the
// K-major tile, zero outside [0, R) x [0, K).
template <int KC>
__device__ __forceinline__ void stage_tile(uint8_t *s, const bf16 *X, long long sr, long long sk, int R, int K, int r0,
                                           int k0) {
    const bf16 zero = __float2bfloat16(0.f);
    const bool rows_fast = sr == 1;  // rows contiguous: consecutive threads take consecutive rows
    for (int t = threadIdx.x; t < GT * KC; t += blockDim.x) {
        const int r = rows_fast ? t % GT : t / KC, k = rows_fast ? t / GT : t % KC;
        const int gr = r0 + r, gk = k0 + k;
        bf16 v = (gr < R && gk < K) ? X[(long long)gr * sr + (long long)gk * sk] : zero;
        *(bf16 *)(s + kmajor_off(r, k, KC)) = v;
    }
}

// The same tile from an FP32 matrix as two BF16 pieces: hi = bf16(x) into s,
// lo = bf16(x - hi) into s + lo_off (x = hi + lo to about 2^-16 |x|).
template <int KC>
__device__ __forceinline__ void stage_tile_split(uint8_t *s, int lo_off, const float *X, long long sr, long long sk,
                                                 int R, int K, int r0, int k0) {
    const bool rows_fast = sr == 1;
    for (int t = threadIdx.x; t < GT * KC; t += blockDim.x) {
        const int r = rows_fast ? t % GT : t / KC, k = rows_fast ? t / GT : t % KC;
        const int gr = r0 + r, gk = k0 + k;
        const float x = (gr < R && gk < K) ? X[(long long)gr * sr + (long long)gk * sk] : 0.f;
        const bf16 hi = __float2bfloat16(x);
        const bf16 lo = __float2bfloat16(x - __bfloat162float(hi));
        *(bf16 *)(s + kmajor_off(r, k, KC)) = hi;
        *(bf16 *)(s + lo_off + kmajor_off(r, k, KC)) = lo;
    }
}

// C[M x N] = A[M x K] * B[N x K]^T on tcgen05, one 128 x 128 tile per block,
// K in stages over a ring of two buffers: the tiles of stage c + 1 are
// staged while the MMAs of stage c run.  SPLIT: A and B are FP32, each staged
// as BF16 hi + lo pieces, and hi*hi + hi*lo + lo*hi accumulate (products of
// about 16-bit operands; the dropped lo*lo is 2^-16 relative).
template <bool SPLIT>
__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
    constexpr int KC = SPLIT ? 32 : GKC;     // K per stage
    constexpr int TILE = GT * KC * 2;         // bytes of one BF16 tile
    constexpr int STAGE = (SPLIT ? 4 : 2) * TILE;  // A, B (then A lo, B lo)
    extern __shared__ __align__(1024) uint8_t dsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5;
    const int m0 = blockIdx.x * GT, n0 = blockIdx.y * GT;
    if (warp == 0) tmem_alloc(&tslot, GT);
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = idesc_bf16_f32(GT, GT);
    bool ok = true;
    const int nk = (g.K + KC - 1) / KC;
    for (int c = 0; c < nk; c++) {
        const int b = c & 1;
        uint8_t *sA = dsm + b * STAGE, *sB = sA + TILE;
        // the MMAs of stage c - 2 (same buffer) must be done before it is refilled
        if (c >= 2) ok = mbar_wait(&mbar[b], (uint32_t)(((c - 2) >> 1) & 1), g.wait) && ok;
        if (SPLIT) {
            stage_tile_split<KC>(sA, 2 * TILE, g.Af, g.sam, g.sak, g.M, g.K, m0, c * KC);
            stage_tile_split<KC>(sB, 2 * TILE, g.Bf, g.sbn, g.sbk, g.N, g.K, n0, c * KC);
        } else {
            stage_tile<KC>(sA, g.A, g.sam, g.sak, g.M, g.K, m0, c * KC);
            stage_tile<KC>(sB, g.B, g.sbn, g.sbk, g.N, g.K, n0, c * KC);
        }
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < KC / 16; kk++) {
                const uint64_t ad = smem_desc(smem_u32(sA) + kk * 256, 128, (KC / 8) * 128);
                const uint64_t bd = smem_desc(smem_u32(sB) + kk * 256, 128, (KC / 8) * 128);
                tc_mma_bf16(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                if (SPLIT) {
                    const uint64_t adl = smem_desc(smem_u32(sA) + 2 * TILE + kk * 256, 128, (KC / 8) * 128);
                    const uint64_t bdl = smem_desc(smem_u32(sB) + 2 * TILE + kk * 256, 128, (KC / 8) * 128);
                    tc_mma_bf16(tmem, ad, bdl, idesc, 1u);
                    tc_mma_bf16(tmem, adl, bd, idesc, 1u);
                }
            }
            tc_commit(&mbar[b]);
        }
    }
    // the last commit completes when every MMA of the tile has
    if (nk > 0) ok = mbar_wait(&mbar[(nk - 1) & 1], (uint32_t)(((nk - 1) >> 1) & 1), g.wait) && ok;
    tc_fence_after();
    __syncthreads();
    if (!ok && g.err) atomicExch(g.err, 1);
    // epilogue: thread = one row of the tile (TMEM lane)
    const int m = m0 + threadIdx.x;
    for (int c0 = 0; c0 < GT; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (m < g.M && nk > 0) {
#pragma unroll
            for (int j = 0; j < 16; j++) {
                int n = n0 + c0 + j;
                if (n >= g.N) break;
                float x = v[j];
                if (g.bias) x += g.bias[n];
                if (g.epi == EPI_BIAS_GELU) {
                    const float h = gelu(x);
                    g.out[(long long)m * g.ldo + n] = x;
                    g.outb[(long long)m * g.ldb + n] = __float2bfloat16(h);
                    if (g.outh) g.outh[(long long)m * g.ldo + n] = h;
                } else if (g.epi == EPI_GELU_BWD) {
                    float d = x * gelu_grad(g.zin[(long long)m * g.ldz + n]);
                    g.out[(long long)m * g.ldo + n] = d;
                    if (g.outb) g.outb[(long long)m * g.ldb + n] = __float2bfloat16(d);
                } else {
                    g.out[(long long)m * g.ldo + n] = x;
                    if (g.outb) g.outb[(long long)m * g.ldb + n] = __float2bfloat16(x);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, GT);
}

// split: FP32 operands in two BF16 pieces (g.Af, g.Bf), three products
static cudaError_t gemm(GemmArgs g, unsigned long long wait, cudaStream_t s, bool split = false) {
    g.wait = wait;
    dim3 grid((g.M + GT - 1) / GT, (g.N + GT - 1) / GT);
    const int smem = split ? 2 * 4 * GT * 32 * 2 : 2 * 2 * GT * GKC * 2;  // 128 KB / 64 KB
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gemm_bf16<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4 * GT * 32 * 2);
        cudaFuncSetAttribute(k_gemm_bf16<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 2 * GT * GKC * 2);
        attr = true;
    }
    if (split)
        k_gemm_bf16<true><<<grid, 128, smem, s>>>(g);
    else
        k_gemm_bf16<false><<<grid, 128, smem, s>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------- small kernels
// splitmix64 (Steele, Lea, Flood 2014) for the seeded initialisation.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

struct MlpLayout {
    long long w1, b1, w2, b2, w3, b3, w4, b4, n;
};

__host__ __device__ inline MlpLayout mlp_layout(int O) {
    MlpLayout L;
    L.w1 = 0;
    L.b1 = L.w1 + MW * 2;
    L.w2 = L.b1 + MW;
    L.b2 = L.w2 + MW * MW;
    L.w3 = L.b2 + MW;
    L.b3 = L.w3 + MW * MW;
    L.w4 = L.b3 + MW;
    L.b4 = L.w4 + (long long)O * MW;
    L.n = L.b4 + O;
    return L;
}

// Weights and biases of a layer with fan-in f uniform on [-1/sqrt(f), 1/sqrt(f)]:
// the first layer's random biases spread its GELU kinks (at -b/w) across the
// input range, which the oscillating coefficient map needs.
__global__ void k_mlp_init(float *p, int O, unsigned long long seed) {
    MlpLayout L = mlp_layout(O);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.n; i += (long long)gridDim.x * blockDim.x) {
        float fan_in = i < L.w2 ? 2.f : (float)MW;
        float a = rsqrtf(fan_in);
        unsigned long long r = splitmix64(seed ^ (unsigned long long)(i * 0x2545F4914F6CDD1Dull));
        float u = (float)((r >> 40) * (1.0 / 16777216.0));  // [0, 1)
        p[i] = a * (2.f * u - 1.f);
    }
}

// BF16 working copies of the four weight matrices (biases stay FP32).
__global__ void k_mlp_bf16(const float *p, bf16 *pb, int O) {
    MlpLayout L = mlp_layout(O);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.n; i += (long long)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16(p[i]);
}

struct StepState {
    long long step;  // Adam steps taken
    float loss_acc;  // running sum of batch losses in the epoch
    float pad;
};

// batch b of the epoch: rows perm(e, b*B + r) of the training set, where
// perm(e, i) = (a_e * i + c_e) mod n with a_e odd-coprime to n (a bijection).
__global__ void k_gather(const float *X, const float *T, long long n, int O, int B, long long steps_per_epoch,
                         unsigned long long seed, const StepState *ss, float *Xb, float *Tb) {
    long long step = ss->step;
    long long e = step / steps_per_epoch, b = step % steps_per_epoch;
    unsigned long long h = splitmix64(seed + 0x51ull * (unsigned long long)e);
    unsigned long long a = (h % (unsigned long long)n) | 1ull;
    while (true) {  // make a coprime to n (n is at most 2^40 here, so this ends quickly)
        unsigned long long x = a, y = (unsigned long long)n;
        while (y) { unsigned long long t = x % y; x = y; y = t; }
        if (x == 1) break;
        a += 2;
    }
    unsigned long long c = splitmix64(h) % (unsigned long long)n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)B * (O + 2);
         t += (long long)gridDim.x * blockDim.x) {
        long long r = t / (O + 2);
        int col = (int)(t % (O + 2));
        unsigned long long i = (unsigned long long)(b * B + r);
        long long src = (long long)((a * (i % (unsigned long long)n) + c) % (unsigned long long)n);
        if (col < 2) Xb[r * 2 + col] = X[src * 2 + col];
        else Tb[r * O + col - 2] = T[src * O + col - 2];
    }
}

// z1 = x W1^T + b1, h1 = gelu(z1) (W1 rounded to BF16 like the other weights)
__global__ void k_l1_fwd(const float *X, int B, const bf16 *pb, const float *p, int O, float *z1, bf16 *h1,
                         float *h1f) {
    MlpLayout L = mlp_layout(O);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)B * MW;
         t += (long long)gridDim.x * blockDim.x) {
        long long r = t / MW;
        int i = (int)(t % MW);
        float w0 = __bfloat162float(pb[L.w1 + i * 2]), w1 = __bfloat162float(pb[L.w1 + i * 2 + 1]);
        float z = fmaf(w0, X[r * 2], fmaf(w1, X[r * 2 + 1], p[L.b1 + i]));
        z1[t] = z;
        const float h = gelu(z);
        h1[t] = __float2bfloat16(h);
        if (h1f) h1f[t] = h;
    }
}

// Fourier input layer (RB_MLP_FOURIER): a row is a snapshot's parameters
// (q, m); omega = 200 eta^(-3/8) m^(-5/8), eta = q / (1 + q)^2 (the chirp
// family's phase rate) in FP64, and h1[f] = cos(omega tau_f),
// h1[128 + f] = sin(omega tau_f) for tau_f = tau_lo + f dtau, f < 128.  The
// phase is reduced modulo 2 pi in FP64, the sine and cosine taken in FP32.
// The layer has no trained parameters (W1, b1 are unused).
__global__ void k_l1_fourier(const float *X, int B, double tau_lo, double dtau, bf16 *h1, float *h1f) {
    constexpr int NF = MW / 2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)B * NF;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / NF;
        const int f = (int)(t % NF);
        const double q = X[r * 2], m = X[r * 2 + 1];
        const double eta = q / ((1.0 + q) * (1.0 + q));
        const double omega = 200.0 * pow(eta, -0.375) * pow(m, -0.625);
        const double ph = omega * (tau_lo + dtau * f);
        const double red = ph - 6.283185307179586 * rint(ph * 0.15915494309189535);
        float sn, cs;
        sincosf((float)red, &sn, &cs);
        h1[r * MW + f] = __float2bfloat16(cs);
        h1[r * MW + NF + f] = __float2bfloat16(sn);
        if (h1f) {
            h1f[r * MW + f] = cs;
            h1f[r * MW + NF + f] = sn;
        }
    }
}

// dy = 2 (y - t) / B, loss += sum (y - t)^2 / B
__global__ void k_loss(const float *y, const float *T, int B, int O, bf16 *dyb, float *dyf, StepState *ss,
                       float *loss_out) {
    float acc = 0.f;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)B * O;
         t += (long long)gridDim.x * blockDim.x) {
        float d = y[t] - T[t];
        acc = fmaf(d, d, acc);
        float g = 2.f * d / (float)B;
        dyf[t] = g;
        dyb[t] = __float2bfloat16(g);
    }
    double s = block_sum((double)acc);
    if (threadIdx.x == 0) {
        if (ss) atomicAdd(&ss->loss_acc, (float)(s / B));
        if (loss_out) atomicAdd(loss_out, (float)(s / B));
    }
}

// dW1[i][c] = sum_b dz1[b][i] x[b][c], db1[i] = sum_b dz1[b][i]; one block per i.
__global__ void k_l1_bwd(const float *dz1, const float *X, int B, float *g, int O) {
    MlpLayout L = mlp_layout(O);
    int i = blockIdx.x;
    double a0 = 0, a1 = 0, ab = 0;
    for (int r = threadIdx.x; r < B; r += blockDim.x) {
        double d = dz1[(long long)r * MW + i];
        a0 += d * X[r * 2];
        a1 += d * X[r * 2 + 1];
        ab += d;
    }
    a0 = block_sum(a0);
    a1 = block_sum(a1);
    ab = block_sum(ab);
    if (threadIdx.x == 0) {
        g[L.w1 + i * 2] = (float)a0;
        g[L.w1 + i * 2 + 1] = (float)a1;
        g[L.b1 + i] = (float)ab;
    }
}

// column sums of an FP32 (B x ncol) matrix into g[off + col]; one block per column
__global__ void k_colsum(const float *X, int B, int ncol, float *g) {
    int c = blockIdx.x;
    double a = 0;
    for (int r = threadIdx.x; r < B; r += blockDim.x) a += X[(long long)r * ncol + c];
    a = block_sum(a);
    if (threadIdx.x == 0) g[c] = (float)a;
}

// Adam (Kingma & Ba) with a cosine-decayed learning rate, then the BF16 copies.
__global__ void k_adam(float *p, const float *g, float *m1, float *m2, bf16 *pb, long long n, StepState *ss,
                       long long total_steps, float lr0, float b1, float b2, float eps) {
    long long t = ss->step + 1;
    float lr = lr0 * 0.5f * (1.f + cosf(3.14159265358979f * (float)(t - 1) / (float)total_steps));
    float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float a = b1 * m1[i] + (1.f - b1) * gi;
        float v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        float x = p[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
        p[i] = x;
        pb[i] = __float2bfloat16(x);
    }
}

__global__ void k_step_done(StepState *ss) { ss->step += 1; }

__global__ void k_epoch_loss(StepState *ss, float *curve, long long steps_per_epoch) {
    long long e = ss->step / steps_per_epoch - 1;
    if (e >= 0) curve[e] = ss->loss_acc / (float)steps_per_epoch;
    ss->loss_acc = 0.f;
}

}  // namespace rbk

using namespace rbk;

struct rb_mlp {
    rb_ctx *ctx = nullptr;
    unsigned long long wait = 0;  // device wait budget (rb_options.timeout_cycles)
    cudaStream_t stream = nullptr;
    int device = 0;
    int O = 0;
    int Bcap = 0;
    MlpLayout L{};
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    bf16 *pb = nullptr;
    float *Xb = nullptr, *Tb = nullptr, *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *y = nullptr, *dyf = nullptr,
          *dz1 = nullptr, *dz2 = nullptr, *dz3 = nullptr;
    bf16 *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *dyb = nullptr, *dz2b = nullptr, *dz3b = nullptr;
    StepState *ss = nullptr;
    int *err = nullptr;
    void *block = nullptr;
    unsigned flags = 0;                    // RB_MLP_FOURIER, RB_MLP_SPLIT
    double tau_lo = 0.0, dtau = 0.0;       // Fourier input layer
    float *h1f = nullptr, *h2f = nullptr, *h3f = nullptr;  // FP32 activations (split forward)
    char msg[256] = {0};
};


namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// forward on rows [0, B) of (X, z/h buffers); y gets B x O.  With
// RB_MLP_SPLIT the three tensor-core layers take FP32 activations and master
// weights as BF16 hi + lo pieces (three products per K step).
cudaError_t forward(rb_mlp *n, const float *X, int B, float *y, cudaStream_t s) {
    const int O = n->O;
    const MlpLayout &L = n->L;
    const bool split = (n->flags & RB_MLP_SPLIT) != 0;
    if (n->flags & RB_MLP_FOURIER) {
        int gf = (int)((B * (long long)(MW / 2) + 255) / 256);
        if (gf > 4096) gf = 4096;
        k_l1_fourier<<<gf, 256, 0, s>>>(X, B, n->tau_lo, n->dtau, n->h1, split ? n->h1f : nullptr);
    } else {
        int g1 = (int)((B * (long long)MW + 255) / 256);
        if (g1 > 4096) g1 = 4096;
        k_l1_fwd<<<g1, 256, 0, s>>>(X, B, n->pb, n->p, O, n->z1, n->h1, split ? n->h1f : nullptr);
    }
    GemmArgs a{};
    a.M = B; a.N = MW; a.K = MW; a.A = n->h1; a.sam = MW; a.sak = 1; a.B = n->pb + L.w2; a.sbn = MW; a.sbk = 1;
    a.epi = EPI_BIAS_GELU; a.bias = n->p + L.b2; a.out = n->z2; a.ldo = MW; a.outb = n->h2; a.ldb = MW; a.err = n->err;
    a.Af = n->h1f; a.Bf = n->p + L.w2; a.outh = split ? n->h2f : nullptr;
    cudaError_t e = gemm(a, n->wait, s, split);
    if (e != cudaSuccess) return e;
    a.A = n->h2; a.B = n->pb + L.w3; a.bias = n->p + L.b3; a.out = n->z3; a.outb = n->h3;
    a.Af = n->h2f; a.Bf = n->p + L.w3; a.outh = split ? n->h3f : nullptr;
    e = gemm(a, n->wait, s, split);
    if (e != cudaSuccess) return e;
    GemmArgs c{};
    c.M = B; c.N = O; c.K = MW; c.A = n->h3; c.sam = MW; c.sak = 1; c.B = n->pb + L.w4; c.sbn = MW; c.sbk = 1;
    c.epi = EPI_STORE; c.bias = n->p + L.b4; c.out = y; c.ldo = O; c.outb = nullptr; c.err = n->err;
    c.Af = n->h3f; c.Bf = n->p + L.w4;
    return gemm(c, n->wait, s, split);
}

// backward of the batch held in the buffers; gradients into n->g
cudaError_t backward(rb_mlp *n, const float *X, int B, cudaStream_t s) {
    const int O = n->O;
    const MlpLayout &L = n->L;
    // dW4 = dy^T h3
    GemmArgs a{};
    a.M = O; a.N = MW; a.K = B; a.A = n->dyb; a.sam = 1; a.sak = O; a.B = n->h3; a.sbn = 1; a.sbk = MW;
    a.epi = EPI_STORE; a.out = n->g + L.w4; a.ldo = MW; a.err = n->err;
    cudaError_t e = gemm(a, n->wait, s);
    if (e != cudaSuccess) return e;
    // dz3 = (dy W4) * gelu'(z3)
    GemmArgs b{};
    b.M = B; b.N = MW; b.K = O; b.A = n->dyb; b.sam = O; b.sak = 1; b.B = n->pb + L.w4; b.sbn = 1; b.sbk = MW;
    b.epi = EPI_GELU_BWD; b.out = n->dz3; b.ldo = MW; b.outb = n->dz3b; b.ldb = MW; b.zin = n->z3; b.ldz = MW;
    b.err = n->err;
    if ((e = gemm(b, n->wait, s)) != cudaSuccess) return e;
    // dW3 = dz3^T h2
    a.M = MW; a.K = B; a.A = n->dz3b; a.sam = 1; a.sak = MW; a.B = n->h2; a.out = n->g + L.w3;
    if ((e = gemm(a, n->wait, s)) != cudaSuccess) return e;
    // dz2 = (dz3 W3) * gelu'(z2)
    b.K = MW; b.A = n->dz3b; b.sam = MW; b.B = n->pb + L.w3; b.out = n->dz2; b.outb = n->dz2b; b.zin = n->z2;
    if ((e = gemm(b, n->wait, s)) != cudaSuccess) return e;
    // dW2 = dz2^T h1
    a.A = n->dz2b; a.B = n->h1; a.out = n->g + L.w2;
    if ((e = gemm(a, n->wait, s)) != cudaSuccess) return e;
    if (!(n->flags & RB_MLP_FOURIER)) {  // the Fourier input layer has no parameters (their gradient stays 0)
        // dz1 = (dz2 W2) * gelu'(z1)
        b.A = n->dz2b; b.B = n->pb + L.w2; b.out = n->dz1; b.outb = nullptr; b.zin = n->z1;
        if ((e = gemm(b, n->wait, s)) != cudaSuccess) return e;
        k_l1_bwd<<<MW, 256, 0, s>>>(n->dz1, X, B, n->g, O);
    }
    k_colsum<<<MW, 256, 0, s>>>(n->dz2, B, MW, n->g + L.b2);
    k_colsum<<<MW, 256, 0, s>>>(n->dz3, B, MW, n->g + L.b3);
    k_colsum<<<O, 256, 0, s>>>(n->dyf, B, O, n->g + L.b4);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

rb_status rb_mlp_create(rb_ctx *ctx, int n_out, int batch_cap, unsigned long long seed, rb_mlp **out) {
    return rb_mlp_create_ex(ctx, n_out, batch_cap, seed, 0u, 0.0, 0.0, out);
}

rb_status rb_mlp_create_ex(rb_ctx *ctx, int n_out, int batch_cap, unsigned long long seed, unsigned flags,
                           double tau_lo, double tau_hi, rb_mlp **out) {
    if (!ctx || !out || n_out < 1 || n_out > 4096 || batch_cap < 1 || batch_cap > (1 << 20)) return RB_EINVAL;
    if ((flags & ~(unsigned)(RB_MLP_FOURIER | RB_MLP_SPLIT)) ||
        ((flags & RB_MLP_FOURIER) && !(tau_lo >= 0.0 && tau_hi > tau_lo && std::isfinite(tau_hi))))
        return RB_EINVAL;
    *out = nullptr;
    rb_mlp *n = new (std::nothrow) rb_mlp();
    if (!n) return RB_ENOMEM;
    n->flags = flags;
    n->tau_lo = tau_lo;
    n->dtau = (flags & RB_MLP_FOURIER) ? (tau_hi - tau_lo) / (double)(MW / 2 - 1) : 0.0;
    n->ctx = ctx;
    n->wait = rbk::ctx_wait_cycles(ctx);
    n->stream = rbk::ctx_stream(ctx);
    n->device = rbk::ctx_device(ctx);
    n->O = n_out;
    n->Bcap = (batch_cap + GT - 1) / GT * GT;
    n->L = mlp_layout(n_out);
    const long long P = n->L.n, B = n->Bcap, O = n_out;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = al256(off + bytes); return o; };
    size_t o_p = take(P * 4), o_g = take(P * 4), o_m1 = take(P * 4), o_m2 = take(P * 4), o_pb = take(P * 2);
    size_t o_Xb = take(B * 2 * 4), o_Tb = take(B * O * 4), o_z1 = take(B * MW * 4), o_z2 = take(B * MW * 4),
           o_z3 = take(B * MW * 4), o_y = take(B * O * 4), o_dyf = take(B * O * 4), o_dz1 = take(B * MW * 4),
           o_dz2 = take(B * MW * 4), o_dz3 = take(B * MW * 4);
    size_t o_h1 = take(B * MW * 2), o_h2 = take(B * MW * 2), o_h3 = take(B * MW * 2), o_dyb = take(B * O * 2),
           o_dz2b = take(B * MW * 2), o_dz3b = take(B * MW * 2);
    size_t o_ss = take(sizeof(StepState)), o_err = take(4);
    const bool split = (flags & RB_MLP_SPLIT) != 0;
    size_t o_h1f = split ? take(B * MW * 4) : 0, o_h2f = split ? take(B * MW * 4) : 0,
           o_h3f = split ? take(B * MW * 4) : 0;
    cudaSetDevice(n->device);
    if (cudaMalloc(&n->block, off) != cudaSuccess) {
        cudaGetLastError();
        delete n;
        return RB_ENOMEM;
    }
    char *w = (char *)n->block;
    n->p = (float *)(w + o_p); n->g = (float *)(w + o_g); n->m1 = (float *)(w + o_m1); n->m2 = (float *)(w + o_m2);
    n->pb = (bf16 *)(w + o_pb);
    n->Xb = (float *)(w + o_Xb); n->Tb = (float *)(w + o_Tb); n->z1 = (float *)(w + o_z1); n->z2 = (float *)(w + o_z2);
    n->z3 = (float *)(w + o_z3); n->y = (float *)(w + o_y); n->dyf = (float *)(w + o_dyf);
    n->dz1 = (float *)(w + o_dz1); n->dz2 = (float *)(w + o_dz2); n->dz3 = (float *)(w + o_dz3);
    n->h1 = (bf16 *)(w + o_h1); n->h2 = (bf16 *)(w + o_h2); n->h3 = (bf16 *)(w + o_h3); n->dyb = (bf16 *)(w + o_dyb);
    n->dz2b = (bf16 *)(w + o_dz2b); n->dz3b = (bf16 *)(w + o_dz3b);
    n->ss = (StepState *)(w + o_ss);
    n->err = (int *)(w + o_err);
    if (split) {
        n->h1f = (float *)(w + o_h1f);
        n->h2f = (float *)(w + o_h2f);
        n->h3f = (float *)(w + o_h3f);
    }
    cudaStream_t s = n->stream;
    cudaMemsetAsync(n->block, 0, off, s);
    k_mlp_init<<<256, 256, 0, s>>>(n->p, n_out, seed);
    k_mlp_bf16<<<256, 256, 0, s>>>(n->p, n->pb, n_out);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(n->block);
        delete n;
        return RB_ECUDA;
    }
    *out = n;
    return RB_OK;
}

void rb_mlp_destroy(rb_mlp *n) {
    if (!n) return;
    cudaSetDevice(n->device);
    cudaStreamSynchronize(n->stream);
    cudaFree(n->block);
    delete n;
}

long long rb_mlp_num_params(const rb_mlp *n) { return n ? n->L.n : 0; }

rb_status rb_mlp_get_params(rb_mlp *n, float *dst) {
    if (!n || !dst) return RB_EINVAL;
    if (cudaMemcpyAsync(dst, n->p, n->L.n * 4, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess) return RB_ECUDA;
    return RB_OK;
}

rb_status rb_mlp_set_params(rb_mlp *n, const float *src) {
    if (!n || !src) return RB_EINVAL;
    cudaStream_t s = n->stream;
    if (cudaMemcpyAsync(n->p, src, n->L.n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return RB_ECUDA;
    cudaMemsetAsync(n->m1, 0, n->L.n * 4, s);
    cudaMemsetAsync(n->m2, 0, n->L.n * 4, s);
    cudaMemsetAsync(n->ss, 0, sizeof(StepState), s);
    k_mlp_bf16<<<256, 256, 0, s>>>(n->p, n->pb, n->O);
    return cudaGetLastError() == cudaSuccess ? RB_OK : RB_ECUDA;
}

rb_status rb_mlp_infer(rb_mlp *n, const float *X, long long rows, float *Y) {
    if (!n || (rows > 0 && (!X || !Y)) || rows < 0) return RB_EINVAL;
    cudaSetDevice(n->device);
    for (long long r0 = 0; r0 < rows; r0 += n->Bcap) {
        int B = (int)(rows - r0 < n->Bcap ? rows - r0 : n->Bcap);
        if (forward(n, X + r0 * 2, B, Y + r0 * n->O, n->stream) != cudaSuccess) return RB_ECUDA;
    }
    return RB_OK;
}

rb_status rb_mlp_grad(rb_mlp *n, const float *X, const float *T, long long rows, float *grad, float *loss) {
    if (!n || !X || !T || !grad || rows < 1 || rows > n->Bcap) return RB_EINVAL;
    cudaSetDevice(n->device);
    cudaStream_t s = n->stream;
    const int B = (int)rows;
    if (loss) cudaMemsetAsync(loss, 0, 4, s);
    if (forward(n, X, B, n->y, s) != cudaSuccess) return RB_ECUDA;
    k_loss<<<64, 256, 0, s>>>(n->y, T, B, n->O, n->dyb, n->dyf, nullptr, loss);
    if (backward(n, X, B, s) != cudaSuccess) return RB_ECUDA;
    if (cudaMemcpyAsync(grad, n->g, n->L.n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return RB_ECUDA;
    return RB_OK;
}

rb_status rb_mlp_train(rb_mlp *n, const float *X, const float *T, long long rows, int epochs, int batch, double lr,
                       unsigned long long seed, float *loss_curve) {
    if (!n || !X || !T || rows < 1 || epochs < 0 || batch < 1 || batch > n->Bcap || batch > rows || !(lr > 0))
        return RB_EINVAL;
    cudaSetDevice(n->device);
    cudaStream_t s = n->stream;
    const long long spe = rows / batch;  // full batches per epoch
    const long long total = spe * epochs;
    if (total == 0) return RB_OK;
    const int B = batch, O = n->O;
    cudaMemsetAsync(n->ss, 0, sizeof(StepState), s);
    cudaMemsetAsync(n->err, 0, 4, s);
    // capture one training step
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return RB_ECUDA;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int gg = (int)(((long long)B * (O + 2) + 255) / 256);
        if (gg > 2048) gg = 2048;
        k_gather<<<gg, 256, 0, cap>>>(X, T, rows, O, B, spe, seed, n->ss, n->Xb, n->Tb);
        forward(n, n->Xb, B, n->y, cap);
        k_loss<<<64, 256, 0, cap>>>(n->y, n->Tb, B, O, n->dyb, n->dyf, n->ss, nullptr);
        backward(n, n->Xb, B, cap);
        k_adam<<<512, 256, 0, cap>>>(n->p, n->g, n->m1, n->m2, n->pb, n->L.n, n->ss, total, (float)lr, 0.9f, 0.999f,
                                     1e-8f);
        k_step_done<<<1, 1, 0, cap>>>(n->ss);
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    rb_status st = RB_OK;
    if (e == cudaSuccess) {
        for (int ep = 0; ep < epochs && e == cudaSuccess; ep++) {
            for (long long b = 0; b < spe && e == cudaSuccess; b++) e = cudaGraphLaunch(exec, s);
            if (loss_curve && e == cudaSuccess) {
                k_epoch_loss<<<1, 1, 0, s>>>(n->ss, loss_curve, spe);
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snprintf(n->msg, sizeof(n->msg), "rb_mlp_train: %s", cudaGetErrorString(e));
        st = RB_ECUDA;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    int herr = 0;
    cudaMemcpy(&herr, n->err, 4, cudaMemcpyDeviceToHost);
    if (st == RB_OK && herr) st = RB_ETIMEOUT;
    return st;
}

}  // extern "C"
