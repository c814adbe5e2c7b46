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
// mode bit 0: A staged MN-major; bit 1: B staged MN-major; bit 2: for an
// MN-major operand, give the descriptor the K-direction core-matrix stride as
// its leading byte offset (else the M/N-direction stride); bit 3: A staged
// MN-major with the 128-byte swizzle (K-direction atom stride 1024 bytes,
// M-direction stride between the two 64-row halves K * 128 bytes).  Operand
// regions (region_a, region_b bytes) hold every byte either reading can reach;
// A starts on a 1024-byte boundary.
__global__ void __launch_bounds__(128) k_tc_selftest(const __half *__restrict__ A, const __half *__restrict__ B,
                                                     float *__restrict__ D, int N, int K, int mode, int region_a,
                                                     int region_b, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem + ((1024u - (tc::smem_u32(smem) & 1023u)) & 1023u);
    unsigned char *sB = smem + region_a;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + region_b);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
    const bool a_sw = mode & 8, a_mn = (mode & 1) || a_sw, b_mn = mode & 2, lbo_k = mode & 4;

    for (int i = tid; i < region_a / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sA)[i] = 0u;
    for (int i = tid; i < region_b / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sB)[i] = 0u;
    __syncthreads();
    for (int i = tid; i < 128 * K; i += blockDim.x) {
        const int r = i / K, k = i % K;
        const uint32_t off = a_sw ? tc::mn_sw128_offset(r, k, K)
                                  : (a_mn ? tc::mnmajor_offset(r, k, 128) : tc::kmajor_offset(r, k, K));
        *reinterpret_cast<__half *>(sA + off) = A[i];
    }
    for (int i = tid; i < N * K; i += blockDim.x) {
        const int r = i / K, k = i % K;
        *reinterpret_cast<__half *>(sB + (b_mn ? tc::mnmajor_offset(r, k, N) : tc::kmajor_offset(r, k, K))) = B[i];
    }
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
        const uint32_t idesc = tc::idesc_f16(128, N, a_mn, b_mn);
        for (int ks = 0; ks < K / 16; ++ks) {
            uint64_t ad, bd;
            if (a_sw) {   // strides: along K 1024 B (8 rows), along M K * 128 B (64-row halves); a K-step = 16 rows
                const uint32_t sk = 1024, sm = (uint32_t)K * 128;
                ad = tc::smem_desc_sw128(tc::smem_u32(sA) + ks * 2048, lbo_k ? sk : sm, lbo_k ? sm : sk);
            } else if (a_mn) {   // strides: along M 128 B, along K (128/8)*128 B; a K-step of 16 = 2 core matrices along K
                const uint32_t sm = 128, sk = 16 * 128;
                ad = tc::smem_desc(tc::smem_u32(sA) + ks * 2 * sk, lbo_k ? sk : sm, lbo_k ? sm : sk);
            } else {
                ad = tc::smem_desc(tc::smem_u32(sA) + ks * 256, 128, (uint32_t)(K / 8) * 128);
            }
            if (b_mn) {
                const uint32_t sn = 128, sk = (uint32_t)(N / 8) * 128;
                bd = tc::smem_desc(tc::smem_u32(sB) + ks * 2 * sk, lbo_k ? sk : sn, lbo_k ? sn : sk);
            } else {
                bd = tc::smem_desc(tc::smem_u32(sB) + ks * 256, 128, (uint32_t)(K / 8) * 128);
            }
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

extern "C" moff_status moff_tc_selftest(const void *a, const void *b, float *d, int n, int k, int mode,
                                        void *cuda_stream) {
    if (!a || !b || !d) return fail_msg(MOFF_EINVAL, "a, b and d must not be NULL");
    if (n < 32 || n > 256 || n % 32 != 0) return fail_msg(MOFF_EINVAL, "n must be a multiple of 32 in [32, 256]");
    if (k < 16 || k > 256 || k % 16 != 0) return fail_msg(MOFF_EINVAL, "k must be a multiple of 16 in [16, 256]");
    if (mode < 0 || mode > 15) return fail_msg(MOFF_EINVAL, "mode must be in [0, 15]");
    // Each operand region holds its tile; an MN-major operand's region also
    // holds every byte either reading of its two descriptor offsets can reach
    // (below 44 KiB for R <= 128 rows and k <= 64).
    const int mn_bound = 48 * 1024;
    // swizzled A: either reading reaches below 1024 + 2 * (k / 8) * k * 128 + k * 128 bytes (< 80 KiB for k <= 64)
    const int region_a = (mode & 8) ? 80 * 1024 : ((mode & 1) ? mn_bound : ((128 * k * 2 + 1023) & ~1023));
    const int region_b = (mode & 2) ? mn_bound : n * k * 2;
    if ((mode & 9) && k > 64) return fail_msg(MOFF_EINVAL, "MN-major A is limited to k <= 64");
    if ((mode & 2) && (k > 64 || n > 128)) return fail_msg(MOFF_EINVAL, "MN-major B is limited to k <= 64, n <= 128");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const size_t smem = (size_t)region_a + region_b + 64 + 1024;   // + alignment slack for A
    void *perr = nullptr;
    if (cudaGetSymbolAddress(&perr, g_selftest_err) != cudaSuccess)
        return fail_msg(MOFF_ECUDA, "cudaGetSymbolAddress failed");
    int *err = static_cast<int *>(perr);
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return fail_msg(MOFF_ECUDA, "memset failed");
    cudaError_t e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail_msg(MOFF_ECUDA, cudaGetErrorString(e));
    k_tc_selftest<<<1, 128, smem, st>>>(static_cast<const __half *>(a), static_cast<const __half *>(b), d, n, k, mode,
                                        region_a, region_b, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_msg(MOFF_ECUDA, cudaGetErrorString(e));
    int h_err = 0;
    if ((e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail_msg(MOFF_ECUDA, cudaGetErrorString(e));
    if (h_err) return fail_msg(MOFF_ETIMEDOUT, "tensor-core product did not complete within its wait limit");
    return MOFF_OK;
}
