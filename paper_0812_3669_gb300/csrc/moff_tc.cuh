// moff_tc.cuh -- Blackwell (sm_103a) tensor-core building blocks: TMEM
// allocation, shared-memory matrix descriptors, tcgen05.mma (kind::f16, FP32
// accumulate, one CTA), completion through an mbarrier with a bounded wait,
// and TMEM -> register loads.  Inline PTX only.
//
// Operand layout used throughout ("canonical K-major, no swizzle"): a tile of
// R rows x K 16-bit elements is stored as 8x8 core matrices (8 rows of 16
// bytes, 128 contiguous bytes each); core matrix (r/8, k/8) sits at
//     base + (r/8) * SBO + (k/8) * 128
// so the leading-dimension byte offset (between core matrices along K) is 128
// and the stride-dimension byte offset (along rows) is SBO = (K/8) * 128.
// An MN-major tile (rows contiguous for each k; see mnmajor_offset) takes
// the K-direction core-matrix stride as its leading byte offset and the
// row-direction stride (128) as its stride byte offset -- checked on the GPU
// by the self-test, where the opposite reading gives a wrong product.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace moff {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) of a K-major tile with K columns.
__device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Byte offset of element (r, k) of an MN-major tile with R rows: core matrix
// (r/8, k/8) holds, for each of its 8 k, the 16 bytes of 8 consecutive r.
__device__ __forceinline__ uint32_t mnmajor_offset(int r, int k, int R) {
    return (uint32_t)((r >> 3) * 128 + (k >> 3) * (R >> 3) * 128 + (k & 7) * 16 + (r & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), fixed version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (r, k) of an MN-major tile with 128-byte swizzling, as a TMA load
// with SWIZZLE_128B writes it (1024-byte aligned base): 64-row halves one after the other,
// each K rows of 128 bytes (64 consecutive r), the 16-byte chunk index XOR-ed with k % 8.
__device__ __forceinline__ uint32_t mn_sw128_offset(int r, int k, int K) {
    return (uint32_t)((r >> 6) * K * 128 + k * 128 + ((((r & 63) >> 3) ^ (k & 7)) << 4) + (r & 7) * 2);
}

// The same descriptor with the 128-byte swizzle layout (bits 61-63 = 2).  For an MN-major
// operand so laid out, the leading byte offset is the MN-direction stride (between 64-element
// halves) and the stride byte offset the K-direction one (1024 bytes per 8 rows) -- the
// reverse of the unswizzled MN-major reading, checked on the GPU by the self-test.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return smem_desc(saddr, lbo, sbo) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, M x N tile (M = 64 or 128, N a multiple of 16 up to 256).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool a_mn = false, bool b_mn = false) {
    return (1u << 4)                            // D format: F32
           | (0u << 7) | (0u << 10)            // A, B format: F16
           | ((a_mn ? 1u : 0u) << 15)          // A major-ness: 0 K-major, 1 MN-major
           | ((b_mn ? 1u : 0u) << 16)          // B major-ness
           | ((uint32_t)(N >> 3) << 17)        // N / 8
           | ((uint32_t)(M >> 4) << 24);       // M / 16
}

// ---- TMEM (one warp executes alloc/dealloc; the address is written to smem)
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Make generic-proxy shared-memory writes visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// ---- MMA: D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        bool accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}
// Arrive once on the mbarrier when every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(mbar))
                 : "memory");
}

// ---- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` to complete, for at most `max_cycles` SM clock
// cycles.  Returns false on time-out (the caller records an error and
// unwinds instead of spinning forever).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, long long max_cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity)) {
        if (clock64() - t0 > max_cycles) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile(
        "{\n"
        ".reg .b64 st;\n"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n"
        "}\n" ::"r"(smem_u32(mbar))
        : "memory");
}

// Bounded wait that also gives up when another role of the CTA has raised
// `abort` (shared memory), so one time-out unwinds every role.
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t *mbar, uint32_t parity, long long max_cycles,
                                                    volatile int *abort) {
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > max_cycles) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

// ---- TMEM -> registers: this warp's 32 lanes x 32 consecutive FP32 columns.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- TMEM -> registers: this warp's 32 lanes x 16 consecutive FP32 columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- TMA tile load (global -> shared) of one box of a 2-D tensor map, completing
// `bytes` of transaction count on an mbarrier armed with mbar_arrive_expect_tx.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
// Bulk copy (global -> shared, no tensor map) of `bytes` (a multiple of 16; both addresses
// 16-byte aligned) completing that many bytes of transaction count on an mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst_smem, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     dst_smem),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}
// x (innermost, elements) times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(uint32_t dst_smem, const void *tmap, int x, int y, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(dst_smem),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}

// ---- TMA bulk tensor store (shared -> global) of one box of a 4-D tensor map,
// tracked by this thread's bulk async-groups.  Coordinates are in elements,
// innermost first; the innermost one times the element size must be a
// multiple of 16 bytes.
__device__ __forceinline__ void tma_store_4d(const void *tmap, uint32_t src_smem, int x, int y, int z, int w) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];\n" ::"l"(tmap),
                 "r"(src_smem), "r"(x), "r"(y), "r"(z), "r"(w)
                 : "memory");
}
// 2-D variant (shared -> global) of the bulk tensor store.
__device__ __forceinline__ void tma_store_2d(const void *tmap, uint32_t src_smem, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];\n" ::"l"(tmap),
                 "r"(src_smem), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// Wait until at most NPEND of this thread's bulk groups still read shared memory.
template <int NPEND>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(NPEND) : "memory");
}
// Wait until every bulk group of this thread has completed (writes performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Device-side error word written when a bounded wait gives up.
constexpr int kErrWaitTimeout = 1;

}  // namespace tc
}  // namespace moff
