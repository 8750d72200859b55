// Host side of the TMA staging (tensor-map encoding through the driver entry
// point, so the library needs no link-time dependency on the driver library),
// and the self-test of the bounded mbarrier wait.
#include <cuda_runtime.h>

#include <mutex>

#include "tma.cuh"

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// Waits on a barrier whose transaction never arrives: the bounded wait must
// expire, record TC_ERR_TIMEOUT and let the kernel return.
__global__ void k_wait_selftest(int *err, unsigned long long limit_ns) {
    __shared__ alignas(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, 16);  // 16 bytes announced, none sent
    }
    __syncthreads();
    mbar_wait(&bar, 0, err, limit_ns);
}

}  // namespace

int tma_encode_f32_3d(CUtensorMap *map, const void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0,
                      uint32_t b1) {
    EncodeTiled fn = encode_fn();
    if (!fn) return TC_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (b0 * 4) % 16 || b0 > 256 || b1 > 256 || b1 == 0)
        return TC_ERR_INVALID_ARG;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {d0 * 4, d0 * d1 * 4};  // bytes, dims 1 and 2
    const cuuint32_t box[3] = {b0, b1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? TC_OK : TC_ERR_UNSUPPORTED;
}

extern "C" int tc_selftest_wait_timeout(void *stream) {
    int *err = nullptr;
    TC_CUDA(cudaMalloc(&err, sizeof(int)));
    int rc = TC_OK, host = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) rc = TC_ERR_CUDA;
    if (!rc) {
        k_wait_selftest<<<1, 32, 0, s>>>(err, 2000000ull);  // 2 ms limit
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&host, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = TC_ERR_CUDA;
    }
    cudaFree(err);
    return rc ? rc : host;
}
