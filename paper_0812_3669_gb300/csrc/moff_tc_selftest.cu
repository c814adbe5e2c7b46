// moff_tc_selftest.cu -- one tensor-core product through the building blocks
// of moff_tc.cuh (operand staging in the canonical layout, TMEM allocation,
// tcgen05.mma, commit + bounded mbarrier wait, tcgen05.ld), exposed as a
// diagnostic entry point so the blocks the DFT kernels rely on are checked
// against a host reference.
#include <cstdio>

#include "../../include/moff.h"
#include "moff_internal.h"
#include "moff_tc.cuh"

namespace moff {
namespace {

__device__ int g_selftest_err;   // time-out flag of the self-test kernel

// D[128][N] = A[128][K] * B[N][K]^T (FP16 in, FP32 out).  128 threads.
__global__ void __launch_bounds__(128) k_tc_selftest(const __half *__restrict__ A, const __half *__restrict__ B,
                                                     float *__restrict__ D, int N, int K, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                                 // 128 x K
    unsigned char *sB = smem + 128 * K * 2;                   // N x K
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + N * K * 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));

    for (int i = tid; i < 128 * K; i += blockDim.x)
        *reinterpret_cast<__half *>(sA + tc::kmajor_offset(i / K, i % K, K)) = A[i];
    for (int i = tid; i < N * K; i += blockDim.x)
        *reinterpret_cast<__half *>(sB + tc::kmajor_offset(i / K, i % K, K)) = B[i];
    tc::fence_async_smem();
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) {
        tc::tmem_alloc(tslot, ncols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (tid == 0) {
        const uint32_t idesc = tc::idesc_f16(128, N);
        const uint32_t sbo = (uint32_t)(K / 8) * 128;
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = tc::smem_desc(tc::smem_u32(sA) + ks * 256, 128, sbo);
            const uint64_t bd = tc::smem_desc(tc::smem_u32(sB) + ks * 256, 128, sbo);
            tc::mma_f16(tbase, ad, bd, idesc, ks > 0);
        }
        tc::mma_commit(mbar);
    }
    bool ok = tc::mbar_wait_bounded(mbar, 0, 4000000000LL);
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int row = warp * 32 + lane;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (c0 + j < N) D[(long long)row * N + c0 + j] = v[j];
        }
    } else if (tid == 0) {
        atomicExch(err, tc::kErrWaitTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

}  // namespace
}  // namespace moff

using namespace moff;

extern "C" moff_status moff_tc_selftest(const void *a, const void *b, float *d, int n, int k, void *cuda_stream) {
    if (!a || !b || !d) return fail_msg(MOFF_EINVAL, "a, b and d must not be NULL");
    if (n < 32 || n > 256 || n % 32 != 0) return fail_msg(MOFF_EINVAL, "n must be a multiple of 32 in [32, 256]");
    if (k < 16 || k > 256 || k % 16 != 0) return fail_msg(MOFF_EINVAL, "k must be a multiple of 16 in [16, 256]");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const size_t smem = (size_t)(128 + n) * k * 2 + 64;
    void *perr = nullptr;
    if (cudaGetSymbolAddress(&perr, g_selftest_err) != cudaSuccess)
        return fail_msg(MOFF_ECUDA, "cudaGetSymbolAddress failed");
    int *err = static_cast<int *>(perr);
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return fail_msg(MOFF_ECUDA, "memset failed");
    cudaError_t e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail_msg(MOFF_ECUDA, cudaGetErrorString(e));
    k_tc_selftest<<<1, 128, smem, st>>>(static_cast<const __half *>(a), static_cast<const __half *>(b), d, n, k, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_msg(MOFF_ECUDA, cudaGetErrorString(e));
    int h_err = 0;
    if ((e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail_msg(MOFF_ECUDA, cudaGetErrorString(e));
    if (h_err) return fail_msg(MOFF_ETIMEDOUT, "tensor-core product did not complete within its wait limit");
    return MOFF_OK;
}
