// rb_noalloc.cu -- a greedy entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running inside a framework that
// owns every byte of device memory through its own pool, services that must
// not grow their footprint after start-up, and hosts where a device
// allocation could block or fail at an unpredictable moment.  For them,
// rb_greedy_noalloc runs the same greedy kernels as rb_greedy with the
// plain-FP64 sweep (which reads complex128 S directly and needs no N x M copy)
// and keeps all of its scratch -- column norms, error sums, picked flags, the
// IMGS work vector and partial sums, the argmax partials and the loop state --
// in one fixed-size array in device global memory, declared below.  The
// array exists once per GPU that loads this library and stays allocated until
// the process exits.
//
// In host code the symbol g_noalloc_scratch is only a host-side stand-in:
// its device address is obtained with cudaGetSymbolAddress, once per device,
// with that device current, on the first call made for that device.
//
// Every call shares the array and the array keeps the previous call's
// contents; the call clears what has to start at zero (the loop state) and
// the init kernel rewrites the per-column sums.  Two calls whose work
// overlaps on the GPU (different streams or host threads) race on the array.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rb_internal.cuh"

namespace {

constexpr long long kNaMaxN = RB_NOALLOC_MAX_N;
constexpr long long kNaMaxM = RB_NOALLOC_MAX_M;
constexpr long long kNaMaxK = RB_NOALLOC_MAX_KMAX;
constexpr long long kNaChunk = 2048;
constexpr long long kNaMaxChunks = (kNaMaxN + kNaChunk - 1) / kNaChunk;
constexpr long long kNaMaxGrid = 4096;  // sweep / IMGS-dot grid cap (152 SMs x occupancy)

constexpr size_t al(size_t x) { return (x + 511) / 512 * 512; }
constexpr size_t kOffNorm = 0;
constexpr size_t kOffAcc = kOffNorm + al(8 * kNaMaxM);
constexpr size_t kOffPick = kOffAcc + al(8 * kNaMaxM);
constexpr size_t kOffV = kOffPick + al(kNaMaxM);
constexpr size_t kOffHp = kOffV + al(16 * kNaMaxN);
constexpr size_t kOffNp = kOffHp + al(16 * kNaMaxK * kNaMaxChunks);
constexpr size_t kOffBe = kOffNp + al(8 * kNaMaxGrid);
constexpr size_t kOffBi = kOffBe + al(8 * kNaMaxGrid);
constexpr size_t kOffSt = kOffBi + al(8 * kNaMaxGrid);
constexpr size_t kScratchBytes = kOffSt + al(sizeof(rbk::DevState));

static_assert(kScratchBytes < (8u << 20), "no-alloc scratch must stay modest");

}  // namespace

// The scratch array (about 4.7 MB for the limits in rb.h).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_na_mutex;
void *g_na_addr[256];
bool g_na_ready[256];

void set_err(char *buf, size_t len, const char *msg) {
    if (buf && len) {
        strncpy(buf, msg, len - 1);
        buf[len - 1] = 0;
    }
}

}  // namespace

extern "C" rb_status rb_greedy_noalloc(const void *S, long long N, long long M, long long ldS, double tol, int kmax,
                                       const rb_options *opt, rb_result *out, char *errbuf, size_t errlen) {
    char msg[256];
    if (!S || !out || !out->Q || !out->pivots || !out->err_curve) {
        set_err(errbuf, errlen, "rb_greedy_noalloc: null S, result, Q, pivots or err_curve");
        return RB_EINVAL;
    }
    if (N < 1 || M < 1 || ldS < N || kmax < 0 || !(tol >= 0.0) || !std::isfinite(tol) || out->ldQ < N ||
        (out->C && out->ldC < M)) {
        set_err(errbuf, errlen, "rb_greedy_noalloc: bad sizes, leading dimensions or tol");
        return RB_EINVAL;
    }
    if (N > kNaMaxN || M > kNaMaxM || kmax > kNaMaxK) {
        snprintf(msg, sizeof(msg),
                 "rb_greedy_noalloc: N=%lld M=%lld kmax=%d exceed the static scratch limits "
                 "N<=%lld M<=%lld kmax<=%lld; use rb_greedy",
                 N, M, kmax, kNaMaxN, kNaMaxM, kNaMaxK);
        set_err(errbuf, errlen, msg);
        return RB_EINVAL;
    }
    if ((reinterpret_cast<uintptr_t>(S) % 16) || (reinterpret_cast<uintptr_t>(out->Q) % 16) ||
        (out->C && (reinterpret_cast<uintptr_t>(out->C) % 16))) {
        set_err(errbuf, errlen, "rb_greedy_noalloc: complex128 arrays must be 16-byte aligned");
        return RB_EINVAL;
    }
    double kappa = opt ? opt->imgs_kappa : 2.0;
    int max_passes = opt ? opt->imgs_max_passes : 4;
    int per_sync = opt ? opt->iters_per_sync : 8;
    cudaStream_t sm = opt ? (cudaStream_t)opt->stream : (cudaStream_t)0;
    if (!(kappa > 1.0) || max_passes < 1 || per_sync < 1) {
        set_err(errbuf, errlen, "rb_greedy_noalloc: bad options");
        return RB_EINVAL;
    }
    int period = opt ? opt->recompute_period : 0;
    if (period < 0) {
        set_err(errbuf, errlen, "rb_greedy_noalloc: bad options");
        return RB_EINVAL;
    }
    if (!out->C) period = 0;  // the recompute reads the stored coefficients; without C there is no room for them
    // the caller's current device is put back on every return path
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        set_err(errbuf, errlen, "rb_greedy_noalloc: cannot read the current device");
        return RB_ECUDA;
    }
    struct DeviceGuard {
        int d;
        ~DeviceGuard() { cudaSetDevice(d); }
    } guard{prev};
    int dev = 0;
    cudaError_t e = opt ? cudaSetDevice(opt->device) : cudaSuccess;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        set_err(errbuf, errlen, "rb_greedy_noalloc: cannot select the device");
        return RB_ECUDA;
    }
    char *w = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ready[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(msg, sizeof(msg), "rb_greedy_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                set_err(errbuf, errlen, msg);
                return RB_ECUDA;
            }
            g_na_addr[dev] = p;
            g_na_ready[dev] = true;
        }
        w = (char *)g_na_addr[dev];
    }
    const int G = rbk::sweep_grid(1 /* plain FP64 sweep */, dev);
    if (G > kNaMaxGrid) {
        set_err(errbuf, errlen, "rb_greedy_noalloc: grid larger than the scratch partial arrays");
        return RB_ESTATE;
    }

    rbk::Prob p{};
    p.N = N;
    p.M = M;
    p.ldS = ldS;
    p.ldH = 0;
    p.ldQ = out->ldQ;
    p.ldC = out->ldC;
    p.minNM = N < M ? N : M;
    p.kmax = kmax;
    p.max_passes = max_passes;
    p.chunk = (int)kNaChunk;
    p.nchunk = (int)((N + kNaChunk - 1) / kNaChunk);
    p.tol = tol;
    p.kappa2 = kappa * kappa;
    p.S = (const double2 *)S;
    p.Q = (double2 *)out->Q;
    p.pivots = out->pivots;
    p.err_curve = out->err_curve;
    p.C = (double2 *)out->C;
    p.rdiag = out->rdiag;
    p.norm2 = (double *)(w + kOffNorm);
    p.acc = (double *)(w + kOffAcc);
    p.picked = (unsigned char *)(w + kOffPick);
    p.v = (double2 *)(w + kOffV);
    p.hpart = (double2 *)(w + kOffHp);
    p.npart = (double *)(w + kOffNp);
    p.bpart_err = (double *)(w + kOffBe);
    p.bpart_idx = (long long *)(w + kOffBi);
    p.st = (rbk::DevState *)(w + kOffSt);

    int nlaunch = 0;
#define NA_CK(call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            snprintf(msg, sizeof(msg), "rb_greedy_noalloc: %s", cudaGetErrorString(e_)); \
            set_err(errbuf, errlen, msg);                                                \
            return RB_ECUDA;                                                             \
        }                                                                                \
    } while (0)
    // the loop state (including the last-block tickets) must start at zero
    NA_CK(cudaMemsetAsync(p.st, 0, sizeof(rbk::DevState), sm));
    NA_CK(rbk::launch_norms(p.S, N, M, ldS, p.norm2, sm));
    NA_CK(rbk::launch_init(p, G, sm));
    nlaunch += 2;
    const int kcap = kmax > 0 ? kmax : 1;
    rbk::DevState hs;
    int it = 0;
    for (;;) {
        for (int t = 0; t < per_sync && it < kcap; t++, it++) {
            NA_CK(rbk::launch_imgs(p, G, false, sm, &nlaunch));
            if (period > 0) {  // the periodic exact recompute, as in rb_greedy
                NA_CK(rbk::launch_recompute(p, period, G, sm));
                nlaunch += 1;
            }
            NA_CK(rbk::launch_sweep(p, 1, G, sm));
            nlaunch += 1;
        }
        NA_CK(cudaMemcpyAsync(&hs, p.st, sizeof(hs), cudaMemcpyDeviceToHost, sm));
        NA_CK(cudaStreamSynchronize(sm));
        if (hs.stop) break;
        if (it >= kcap) {
            set_err(errbuf, errlen, "rb_greedy_noalloc: loop did not stop after kmax iterations");
            return RB_ESTATE;
        }
    }
    if (out->final_err) {
        NA_CK(rbk::launch_final_err(p, out->final_err, sm));
        nlaunch += 1;
    }
    NA_CK(cudaStreamSynchronize(sm));
#undef NA_CK
    out->k = hs.k;
    out->status = hs.status;
    out->imgs_passes = hs.total_passes;
    out->switch_iter = -1;
    out->n_launches = nlaunch;
    out->n_sweeps = hs.n_sweeps;
    out->ms_total = 0.0;
    out->ms_sweep = 0.0;
    out->sweep_bytes = (double)hs.n_sweeps * (16.0 * N * M + 16.0 * N + 41.0 * M);
    if (hs.status < 0) {
        set_err(errbuf, errlen,
                hs.status == RB_ENONFINITE ? "rb_greedy_noalloc: NaN or Inf in S"
                : hs.status == RB_EORTHO   ? "rb_greedy_noalloc: IMGS did not pass the kappa test"
                                           : "rb_greedy_noalloc: device error");
    }
    return (rb_status)hs.status;
}
