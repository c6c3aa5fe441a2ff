// peaks.cu -- peak-rate probes of one GPU: the denominators of the rooflines
// that the benchmark reports (FP32 FMA pipe, FP64 FMA pipe, TF32 tensor cores).
//
// Each probe is a kernel that does nothing but the operation it measures,
// with enough independent work per SM to hide the pipeline latency; the host
// side times repeated launches with CUDA events and keeps the best rate.
#include "pdilqr_bench.h"

#include <algorithm>

#include "dev_linalg.cuh"

using namespace pdl;

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kUnroll = 16;   // FMAs per chain per loop trip

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, T b, T c, int iters)
{
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + blockIdx.x) * (T)1e-7 + (T)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    // practically never true: keeps the chains alive without a store per thread
    if (s == (T)-1234.5) out[blockIdx.x] = s;
}

// TF32 tensor-core probe: one CTA per SM; thread 0 issues `count` MMAs of
// M = 128, N = 256, K = 8 (kind::tf32, FP32 accumulators in TMEM) on fixed
// shared-memory tiles, commits them to an mbarrier, and the CTA waits for
// completion with a bounded wait (err[0] is set if it runs out).
constexpr int kTcN = 256;
constexpr int kOneCtaSmem = 160 * 1024;

// (launched with a large dynamic shared-memory request that keeps one CTA per SM)
__global__ void __launch_bounds__(128) tf32_probe_kernel(int count, int* err)
{
    __shared__ __align__(1024) float a_tile[128 * 8];
    __shared__ __align__(1024) float b_tile[kTcN * 8];
    __shared__ TcCtx tc;
    for (int e = threadIdx.x; e < 128 * 8; e += blockDim.x) a_tile[e] = 1e-3f * (e & 7);
    for (int e = threadIdx.x; e < kTcN * 8; e += blockDim.x) b_tile[e] = 1e-3f * (e & 3);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_setup(&tc, kTcN);
    constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t da = tc_sdesc(a_tile), db = tc_sdesc(b_tile);
        for (int i = 0; i < count; ++i) tc_mma(tc.tmem, da, db, IDESC, i == 0 ? 0u : 1u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&tc.mbar)) : "memory");
    }
    const bool done = mbar_wait_bounded(&tc.mbar, 0, 2000000000ull);
    const bool failed = __syncthreads_or(done ? 0 : 1) != 0;
    if (failed) {
        if (!done) mbar_wait_bounded(&tc.mbar, 0, kTcDrainNs);
        if (threadIdx.x == 0) atomicExch(err, 1);
    }
    tc_teardown(&tc);
}

struct Timer {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Timer() { cudaEventCreate(&e0); cudaEventCreate(&e1); }
    ~Timer() { cudaEventDestroy(e0); cudaEventDestroy(e1); }
};

}  // namespace

extern "C" pdilqr_status pdilqr_peak_probe(int32_t kind, int32_t reps, double* tflops,
                                           double* ms_out)
{
    if (!tflops || reps < 1 || kind < PDILQR_PEAK_FFMA || kind > PDILQR_PEAK_TF32_MMA)
        return PDILQR_E_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PDILQR_E_CUDA;
    void* buf = nullptr;
    if (cudaMalloc(&buf, 1 << 20) != cudaSuccess) return PDILQR_E_NO_MEMORY;
    int* err = static_cast<int*>(buf);
    cudaMemset(err, 0, sizeof(int));
    if (kind == PDILQR_PEAK_TF32_MMA &&
        cudaFuncSetAttribute(tf32_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kOneCtaSmem) != cudaSuccess) {
        cudaFree(buf);
        return PDILQR_E_CUDA;
    }
    Timer t;
    double flops = 0.0;
    // one launch with `work` units; returns its time in ms
    auto launch = [&](int work) -> float {
        cudaEventRecord(t.e0);
        if (kind == PDILQR_PEAK_FFMA) {
            fma_probe_kernel<float><<<sms * 8, 256>>>(static_cast<float*>(buf) + 64, 0.999999f, 1e-7f, work);
            flops = 2.0 * kChains * kUnroll * (double)work * sms * 8 * 256;
        } else if (kind == PDILQR_PEAK_DFMA) {
            fma_probe_kernel<double><<<sms * 8, 256>>>(static_cast<double*>(buf) + 64, 0.999999, 1e-7, work);
            flops = 2.0 * kChains * kUnroll * (double)work * sms * 8 * 256;
        } else {
            tf32_probe_kernel<<<sms, 128, kOneCtaSmem>>>(work, err);
            flops = 2.0 * 128 * kTcN * 8 * (double)work * sms;
        }
        cudaEventRecord(t.e1);
        cudaEventSynchronize(t.e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.e0, t.e1);
        return ms;
    };
    // size the launch to about 50 ms, then keep the best of `reps`
    int work = 16;
    float ms = launch(work);
    for (int g = 0; g < 20 && ms < 5.f && work < (1 << 26); ++g) ms = launch(work *= 4);
    work = std::max(1, (int)std::min(2.0e9, work * (50.0 / std::max(ms, 1e-3f))));
    double best = 0.0, best_ms = 0.0;
    for (int r = 0; r < reps; ++r) {
        ms = launch(work);
        const double rate = flops / (ms * 1e-3) / 1e12;
        if (rate > best) { best = rate; best_ms = ms; }
    }
    int herr = 0;
    cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    if (e != cudaSuccess) return PDILQR_E_CUDA;
    if (herr) return PDILQR_E_TIMEOUT;
    *tflops = best;
    if (ms_out) *ms_out = best_ms;
    return PDILQR_OK;
}
