// Measured non-tensor FMA throughput of the device: the denominators of the
// pair passes' ALU rooflines (the passes are plain FP32 / FP64 arithmetic,
// no dense contraction).  Every SM runs resident blocks of threads that
// each advance 8 independent FMA chains; the rate is 2 flop per FMA over
// the best of a few CUDA-event-timed launches.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/sph.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

// x <- x * b + c per chain: with b = 1 - 2^-20 and c = 2^-20 the chains
// stay at 1 (no overflow, no subnormals) and nothing folds at compile
// time, since b, c and the start values come from the host.
template <typename R>
__global__ void __launch_bounds__(PROBE_THREADS)
    k_fma_probe(R b, R c, R x0, long long iters, R *sink) {
    R x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = x0 + (R)k * c;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], b, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == (R)-1) sink[threadIdx.x] = s;   // never true: keeps the chains
}

template <typename R>
sph_status probe(cudaStream_t st, double *flops, int *sms_out) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<R>,
                                                      PROBE_THREADS, 0) != cudaSuccess ||
        sms <= 0 || per_sm <= 0) {
        cudaGetLastError();
        return SPH_ECUDA;
    }
    const int blocks = sms * per_sm;
    R *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&sink, sizeof(R) * PROBE_THREADS) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ENOMEM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const R b = (R)1 - (R)9.5367431640625e-07, c = (R)9.5367431640625e-07;
    // size a launch to ~20 ms from a short first one
    long long iters = 1 << 12;
    double best = 0.0;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, st);
        k_fma_probe<R><<<blocks, PROBE_THREADS, 0, st>>>(b, c, (R)1, iters, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double fl = 2.0 * PROBE_CHAINS * (double)iters * blocks * PROBE_THREADS;
        if (rep > 0) best = std::max(best, fl / (ms * 1e-3));
        if (ms > 0.f && ms < 10.f)
            iters = std::min<long long>(iters * std::max(2.0, 20.0 / ms), 1ll << 30);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || best <= 0.0) return SPH_ECUDA;
    *flops = best;
    if (sms_out) *sms_out = sms;
    return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_probe_fma(int fp64, void *stream, double *flops,
                                    int *sms) {
    if (!flops || (fp64 != 0 && fp64 != 1)) return SPH_EINVAL;
    const cudaStream_t st = (cudaStream_t)stream;
    return fp64 ? probe<double>(st, flops, sms) : probe<float>(st, flops, sms);
}
