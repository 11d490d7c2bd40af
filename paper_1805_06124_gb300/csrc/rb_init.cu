// rb_init.cu -- input-side kernels: synthetic snapshots, hi/lo split with
// column norms, and the first argmax of the greedy (Alg. 3, before the loop:
// sigma_0(s_i) = ||s_i||, j(0) = arg sup_i sigma_0(s_i)).
#include "rb_internal.cuh"

namespace rbk {

// t-dependent factors of the chirp: amp_i = (t_c - t_i)^(-1/4),
// ph_i = (t_c - t_i)^(5/8), t_i = i/N, t_c = 1.05.
__global__ void k_generate_tables(double *amp, double *ph, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        double tau = 1.05 - (double)i / (double)N;
        amp[i] = pow(tau, -0.25);
        ph[i] = pow(tau, 0.625);
    }
}

// One block per column (grid-stride): s_j(t_i) = amp_i exp(-i omega_j ph_i),
// then divided by ||s_j||.
__global__ void __launch_bounds__(kThreads) k_generate(const double *q, const double *m, const double *amp,
                                                       const double *ph, long long N, long long M, double2 *S,
                                                       long long ldS) {
    for (long long j = blockIdx.x; j < M; j += gridDim.x) {
        double qq = q[j];
        double eta = qq / ((1.0 + qq) * (1.0 + qq));
        double omega = 200.0 * pow(eta, -0.375) * pow(m[j], -0.625);
        double2 *s = S + j * ldS;
        double nrm = 0.0;
        for (long long i = threadIdx.x; i < N; i += blockDim.x) {
            double sn, cs;
            sincos(omega * ph[i], &sn, &cs);
            double2 val = make_double2(amp[i] * cs, -(amp[i] * sn));
            s[i] = val;
            nrm = fma(val.x, val.x, fma(val.y, val.y, nrm));
        }
        __shared__ double scale;
        double tot = block_sum(nrm);
        if (threadIdx.x == 0) scale = sqrt(tot);
        __syncthreads();
        double d = scale;
        for (long long i = threadIdx.x; i < N; i += blockDim.x) {
            double2 val = s[i];
            s[i] = make_double2(val.x / d, val.y / d);
        }
        __syncthreads();
    }
}

// Warp per column: hi = fl32(x), lo = fl32(x - hi) (round to nearest) and,
// when norm2 != null, ||hi + lo||^2 in double-float: the sweep works on
// hi + lo, so its norms are taken of the same numbers.  Lane L handles the
// element pairs (2t, 2t+1), t = L (mod 32) -- the partition and the steps of
// norm2_acc4, shared with the split form's init -- reading S with two
// 16-byte loads per pair (the second hits L1) and storing hi/lo as float4
// when ldH is even and the arrays are 16-byte aligned.  hi == null: norms
// only (columns that stay in host memory).
__global__ void __launch_bounds__(kThreads) k_split(const double2 *__restrict__ S, long long N, long long M,
                                                    long long ldS, float2 *__restrict__ hi,
                                                    float2 *__restrict__ lo, long long ldH,
                                                    double *__restrict__ norm2) {
    int lane = threadIdx.x & 31;
    long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long n2 = N >> 1;
    const bool vec = hi && !(ldH & 1) && !(reinterpret_cast<uintptr_t>(hi) & 15) &&
                     !(reinterpret_cast<uintptr_t>(lo) & 15);
    for (long long j = gw; j < M; j += nw) {
        const double2 *s = S + j * ldS;
        float2 *h = hi ? hi + j * ldH : nullptr;
        float2 *l = hi ? lo + j * ldH : nullptr;
        Norm2Acc a{0.f, 0.f, 0.f};
        constexpr int U = 2;
        for (long long t = lane; t < n2; t += 32 * U) {
            double2 x[2 * U];
#pragma unroll
            for (int u = 0; u < U; u++)
                if (t + 32 * u < n2) {
                    x[2 * u] = __ldg(s + 2 * (t + 32 * u));
                    x[2 * u + 1] = __ldg(s + 2 * (t + 32 * u) + 1);
                }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const long long tu = t + 32 * u;
                if (tu >= n2) break;
                float2 h0, l0, h1, l1;
                split_c(x[2 * u], h0, l0);
                split_c(x[2 * u + 1], h1, l1);
                const float4 hv = make_float4(h0.x, h0.y, h1.x, h1.y);
                const float4 lv = make_float4(l0.x, l0.y, l1.x, l1.y);
                if (vec) {
                    reinterpret_cast<float4 *>(h)[tu] = hv;
                    reinterpret_cast<float4 *>(l)[tu] = lv;
                } else if (h) {
                    h[2 * tu] = h0;
                    h[2 * tu + 1] = h1;
                    l[2 * tu] = l0;
                    l[2 * tu + 1] = l1;
                }
                norm2_acc4(a, hv, lv);
            }
        }
        if ((N & 1) && lane == 0) {
            float2 h0, l0;
            split_c(__ldg(s + N - 1), h0, l0);
            if (h) {
                h[N - 1] = h0;
                l[N - 1] = l0;
            }
            norm2_acc2(a, h0, l0);
        }
        if (norm2) {
            const double nrm = norm2_finish(a);
            if (lane == 0) norm2[j] = nrm;
        }
    }
}

// Warp per column: ||s_j||^2 in FP64 straight from complex128 (plain-FP64 form).
__global__ void __launch_bounds__(kThreads) k_norms(const double2 *__restrict__ S, long long N, long long M,
                                                    long long ldS, double *__restrict__ norm2) {
    int lane = threadIdx.x & 31;
    long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long j = gw; j < M; j += nw) {
        const double2 *s = S + j * ldS;
        double nrm = 0.0;
        for (long long i = lane; i < N; i += 32) {
            double2 x = ld_stream_d2(s + i);
            nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
        }
        nrm = warp_sum(nrm);
        if (lane == 0) norm2[j] = nrm;
    }
}

// acc_j = 0, picked_j = 0, first pivot = argmax ||s_j||^2, err_curve[0].
__global__ void __launch_bounds__(kThreads) k_init(Prob p) {
    DevState *st = p.st;
    double be = -INFINITY;
    long long bi = kNoIdx;
    int bad = 0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p.M;
         j += (long long)gridDim.x * blockDim.x) {
        double e = p.norm2[j];
        p.acc[j] = 0.0;
        p.picked[j] = 0;
        if (!isfinite(e)) bad = 1;
        if (better(e, j, be, bi)) { be = e; bi = j; }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->nonfinite, 1);
    block_best(be, bi);
    if (threadIdx.x == 0) {
        p.bpart_err[blockIdx.x] = be;
        p.bpart_idx[blockIdx.x] = bi;
    }
    if (!last_block(&st->ticket_init)) return;
    be = -INFINITY;
    bi = kNoIdx;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        double e = __ldcg(p.bpart_err + b);
        long long i = __ldcg(p.bpart_idx + b);
        if (better(e, i, be, bi)) { be = e; bi = i; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        st->ticket_init = 0;
        st->k = 0;
        st->switch_iter = -1;
        double emax = bi == kNoIdx ? 0.0 : be;
        p.err_curve[0] = emax;
        st->J = bi;
        st->errJ = emax;
        if (ld_volatile(&st->nonfinite)) {
            st->status = RB_ENONFINITE;
            st->stop = 1;
        } else if (bi == kNoIdx || emax < p.tol) {
            st->status = RB_OK;
            st->stop = 1;
        } else if (p.kmax <= 0) {
            st->status = RB_KMAX_REACHED;
            st->stop = 1;
        }
    }
}

// Resume from a checkpoint of k0 basis vectors (Q rows, pivots and C rows
// 0..k0-1 given): acc_j is rebuilt from C with error-free squares and a
// compensated sum (the k_recompute formula), picked is cleared, and norms are
// checked.
__global__ void __launch_bounds__(kThreads) k_resume_acc(Prob p, int k0) {
    DevState *st = p.st;
    int bad = 0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p.M;
         j += (long long)gridDim.x * blockDim.x) {
        double s = 0.0, e = 0.0;
        for (int l = 0; l < k0; l++) {
            const double2 c = p.C[(long long)l * p.ldC + j];
            const double x = c.x * c.x, ex = fma(c.x, c.x, -x);
            const double y = c.y * c.y, ey = fma(c.y, c.y, -y);
            double t = s + x, b = t - s;
            e += ((s - (t - b)) + (x - b)) + ex;
            s = t;
            t = s + y;
            b = t - s;
            e += ((s - (t - b)) + (y - b)) + ey;
            s = t;
        }
        p.acc[j] = s + e;
        p.picked[j] = 0;
        if (!isfinite(p.norm2[j]) || !isfinite(s + e)) bad = 1;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->nonfinite, 1);
}

// Mark the checkpoint's pivots (validated on the host: distinct, in [0, M)).
__global__ void k_resume_mark(Prob p, int k0) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < k0; l += gridDim.x * blockDim.x) p.picked[p.pivots[l]] = 1;
}

// After k_resume_mark: the argmax of err_j = ||s_j||^2 - acc_j over unpicked
// columns, err_curve[k0], the next pivot and the stopping rule, as the last
// block of a sweep would leave them after iteration k0 - 1.
__global__ void __launch_bounds__(kThreads) k_resume_pick(Prob p, int k0) {
    DevState *st = p.st;
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p.M;
         j += (long long)gridDim.x * blockDim.x) {
        const double e = p.norm2[j] - p.acc[j];
        if (!p.picked[j] && better(e, j, be, bi)) {
            be = e;
            bi = j;
        }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        p.bpart_err[blockIdx.x] = be;
        p.bpart_idx[blockIdx.x] = bi;
    }
    if (!last_block(&st->ticket_init)) return;
    be = -INFINITY;
    bi = kNoIdx;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        double e = __ldcg(p.bpart_err + b);
        long long i = __ldcg(p.bpart_idx + b);
        if (better(e, i, be, bi)) { be = e; bi = i; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        st->ticket_init = 0;
        st->k = k0;
        st->switch_iter = -1;
        const double emax = bi == kNoIdx ? 0.0 : be;
        p.err_curve[k0] = emax;
        st->J = bi;
        st->errJ = emax;
        if (ld_volatile(&st->nonfinite)) {
            st->status = RB_ENONFINITE;
            st->stop = 1;
        } else if (bi == kNoIdx || emax < p.tol) {
            st->status = RB_OK;
            st->stop = 1;
        } else if (k0 >= p.kmax) {
            st->status = RB_KMAX_REACHED;
            st->stop = 1;
        } else if (k0 >= p.minNM) {
            st->status = RB_OK;
            st->stop = 1;
        }
    }
}

__global__ void k_final_err(Prob p, double *final_err) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p.M;
         j += (long long)gridDim.x * blockDim.x)
        final_err[j] = p.norm2[j] - p.acc[j];
}

static int grid_for(long long work, int threads, int cap) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

cudaError_t launch_generate_tables(double *amp, double *ph, long long N, cudaStream_t s) {
    k_generate_tables<<<grid_for(N, kThreads, 4096), kThreads, 0, s>>>(amp, ph, N);
    return cudaGetLastError();
}

cudaError_t launch_generate(const double *q, const double *m, const double *amp, const double *ph, long long N,
                            long long M, double2 *S, long long ldS, cudaStream_t s) {
    int g = (int)(M < 152 * 16 ? M : 152 * 16);
    k_generate<<<g, kThreads, 0, s>>>(q, m, amp, ph, N, M, S, ldS);
    return cudaGetLastError();
}

cudaError_t launch_split(const double2 *S, long long N, long long M, long long ldS, float2 *hi, float2 *lo,
                         long long ldH, double *norm2, cudaStream_t s) {
    int g = grid_for(M * 32, kThreads, 152 * 8);
    k_split<<<g, kThreads, 0, s>>>(S, N, M, ldS, hi, lo, ldH, norm2);
    return cudaGetLastError();
}

cudaError_t launch_norms(const double2 *S, long long N, long long M, long long ldS, double *norm2,
                         cudaStream_t s) {
    int g = grid_for(M * 32, kThreads, 152 * 8);
    k_norms<<<g, kThreads, 0, s>>>(S, N, M, ldS, norm2);
    return cudaGetLastError();
}

cudaError_t launch_init(const Prob &p, int grid, cudaStream_t s) {
    int g = grid_for(p.M, kThreads, grid);
    k_init<<<g, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_resume(const Prob &p, int k0, int grid, cudaStream_t s) {
    const int g = grid_for(p.M, kThreads, grid);
    k_resume_acc<<<g, kThreads, 0, s>>>(p, k0);
    k_resume_mark<<<(k0 + 255) / 256, 256, 0, s>>>(p, k0);
    k_resume_pick<<<g, kThreads, 0, s>>>(p, k0);
    return cudaGetLastError();
}

cudaError_t launch_final_err(const Prob &p, double *final_err, cudaStream_t s) {
    k_final_err<<<grid_for(p.M, kThreads, 4096), kThreads, 0, s>>>(p, final_err);
    return cudaGetLastError();
}

}  // namespace rbk
