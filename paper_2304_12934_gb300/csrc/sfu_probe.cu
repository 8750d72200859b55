// Throughput of the special-function unit for lg2, ex2 and rcp, measured on
// the device at hand: the roof of the prior kernel, whose pair evaluations
// take one of each per cell (Sec. 3 Eqs. reg2, reg3 through rho').  Each
// thread runs independent dependency chains of one operation (plus one FMA-
// pipe operation per step, which runs at several times the rate), enough
// warps and chains to keep the unit busy; nothing is allocated.
#include "common.cuh"
#include "sfu.cuh"

namespace {

constexpr int kChains = 8, kIters = 2048, kThreads = 256, kBlocksPerSM = 8, kReps = 5;

__device__ float g_sfu_sink;

template <int OP>
__global__ void __launch_bounds__(kThreads) k_sfu_probe(float seed) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + 0.01f * c + 1e-6f * threadIdx.x;
#pragma unroll 1
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) v[c] = lg2a(v[c]) + 2.0f;   // stays near its fixed point 4
            if (OP == 1) v[c] = ex2a(v[c]) * 0.25f;  // near 0.31
            if (OP == 2) v[c] = rcpa(v[c]) + 0.5f;   // near 1.28
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.0f) g_sfu_sink = s;  // never true; keeps the chains alive
}

template <int OP>
int time_probe(int blocks, cudaStream_t s, float *ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    TC_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return TC_ERR_CUDA;
    }
    for (int w = 0; w < 2; ++w) k_sfu_probe<OP><<<blocks, kThreads, 0, s>>>(1.5f);
    cudaEventRecord(a, s);
    for (int r = 0; r < kReps; ++r) k_sfu_probe<OP><<<blocks, kThreads, 0, s>>>(1.5f);
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return tc_cuda_fail(e, "k_sfu_probe");
    return TC_OK;
}

}  // namespace

extern "C" int tc_sfu_throughput(int op, double *lane_ops_per_s, void *stream) {
    if (op < 0 || op > 2 || !lane_ops_per_s) return TC_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    TC_CUDA(cudaGetDevice(&dev));
    TC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * kBlocksPerSM;
    cudaStream_t s = (cudaStream_t)stream;
    float ms = 0.f;
    const int rc = op == 0 ? time_probe<0>(blocks, s, &ms) : op == 1 ? time_probe<1>(blocks, s, &ms)
                                                                    : time_probe<2>(blocks, s, &ms);
    if (rc) return rc;
    TC_LAUNCHED("k_sfu_probe");
    if (!(ms > 0.f)) return TC_ERR_CUDA;
    *lane_ops_per_s = (double)blocks * kThreads * kChains * kIters * kReps / (ms * 1e-3);
    return TC_OK;
}
