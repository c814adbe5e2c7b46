// moff_gridtc.cu -- Eq. m6 step 2 (the gridding W^T) of Morales (arXiv
// 0812.3669) for dense arrays on the 5th-generation tensor cores.
//
// The gridded field of one tile of 8 x 8 cells is a linear map of the weighted
// voltages of the antennas whose kernels reach the tile:
//     G(t, p_out, cell) = sum_{a, p_in} W_{a, p_out, p_in}(cell - anchor_a) y_{t, a, p_in},
// a small dense product per tile: [128 samples x K] (the voltages, K = 2 x the
// tile's antenna-pols, real and imaginary parts) times [K x 2 P 64] (the tile's
// kernel values in real form).  Antennas are numbered in raster order of their
// anchor cells, so the antennas of one anchor row that reach a tile are
// consecutive voltage-plane rows: a tile's K is a few runs of plane rows, cut
// into chunks of 16 rows (one TMA box each of the real and imaginary planes).
// Slots of a chunk past its run's end read other voltages against zero kernel
// values.
//
//   k_grid_tc  one CTA per (tile, channel group): the tile's kernel matrix B is
//              resident in shared memory (FP16, scaled by the plan's power of two
//              so that |G| stays in range); for every channel of the group and
//              block of 128 samples, one lane streams the chunks of A by TMA
//              (128-byte swizzle, MN-major), one lane issues tcgen05.mma into one
//              of two TMEM accumulators, and eight warps convert the accumulator
//              to FP16 and store the tile's field rows [re 8][im 8] per (pol, row).
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "moff_internal.h"
#include "moff_tc.cuh"

namespace moff {
namespace {

constexpr int kGtEpiWarps = 8;
constexpr int kGtThreads = (kGtEpiWarps + 2) * 32;
constexpr int kGtMaxStages = 8;                          // A ring depth: as many as shared memory allows, <= 8
constexpr int kGtChunkRows = 16;                         // plane rows per chunk
constexpr int kGtChunkK = 2 * kGtChunkRows;              // contraction per chunk (re rows, im rows)
constexpr int kGtStageBytes = 128 * kGtChunkK * 2;       // 128 samples x 32 k, FP16
constexpr int kGtHalfBytes = kGtStageBytes / 2;          // one 64-sample half: 32 k-rows x 128 bytes
constexpr long long kGtWaitCycles = 200000000LL;         // ~0.1 s at the SM clock
constexpr int kGtBoxBytes = 32 * 128;                    // epilogue box: 32 samples x 64 halves, 128-byte swizzle

template <int P>
__global__ void __launch_bounds__(kGtThreads, 1)
    k_grid_tc(const GridTcArgs a, const __grid_constant__ CUtensorMap amap_re,
              const __grid_constant__ CUtensorMap amap_im, const __grid_constant__ CUtensorMap gmap) {
    constexpr int NT = 128 * P;                           // output columns (p, cy, re/im, cx)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int item = blockIdx.x;
    const int tcell = a.tile_cell[item];
    const int ty = tcell >> 16, tx = tcell & 0xFFFF;
    const int kp = a.kp[item];
    const int ch0 = a.chunk_off[item];
    const int nchunk = kp / kGtChunkK;

    const int cper = (a.nc + gridDim.y - 1) / gridDim.y;
    const int cb = blockIdx.y * cper, ce = min(a.nc, cb + cper);
    if (cb >= ce) return;
    const int ntb = (a.nt + 127) / 128;
    const int nitems = (ce - cb) * ntb;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const size_t bbytes = ((size_t)NT * a.kp_max * 2 + 1023) & ~(size_t)1023;
    unsigned char *sB = smem;                                  // NT x kp, K-major (resident)
    const int ns = a.stages;
    unsigned char *sA = sB + bbytes;                           // ns x [128 x 32], 1024-aligned
    unsigned char *sE = sA + ns * kGtStageBytes;               // a.boxes epilogue boxes per warp, 1024-aligned
    uint64_t *bars = reinterpret_cast<uint64_t *>(sE + kGtEpiWarps * a.boxes * kGtBoxBytes);
    uint64_t *a_full = bars, *a_empty = bars + ns, *d_full = bars + 2 * ns, *d_empty = bars + 2 * ns + 2,
             *b_full = bars + 2 * ns + 4;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * ns + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const uint32_t bbytes_item = (uint32_t)(NT * kp * 2);

    if (tid == 0) {
        for (int s = 0; s < ns; ++s) {
            tc::mbar_init(&a_full[s], 1);
            tc::mbar_init(&a_empty[s], 1);
        }
        tc::mbar_init(b_full, 1);
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&d_full[b], 1);
            tc::mbar_init(&d_empty[b], kGtEpiWarps * 32);
        }
        *abort_flag = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, 2 * NT);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == kGtEpiWarps) {
        // ---------------- producer (one lane): the tile's kernel matrix B by one bulk copy
        // (completing on b_full), then chunk g into stage g % ns, four TMA boxes (re / im rows x
        // two 64-sample halves) completing on a_full
        if (lane == 0) {
            tc::mbar_arrive_expect_tx(b_full, bbytes_item);
            tc::bulk_load(tc::smem_u32(sB), reinterpret_cast<const unsigned char *>(a.bimg) + a.bimg_off[item],
                          bbytes_item, b_full);
            int g = 0;
            for (int i = 0; i < nitems && !*abort_flag; ++i) {
                const int cl = cb + i / ntb, t0b = (i % ntb) * 128;
                bool ok = true;
                for (int ch = 0; ch < nchunk; ++ch, ++g) {
                    const int st = g % ns;
                    if (!tc::mbar_wait_abortable(&a_empty[st], (uint32_t)(((g / ns) & 1) ^ 1), kGtWaitCycles,
                                                 abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = tc::smem_u32(sA + st * kGtStageBytes);
                    const int y = cl * a.AP + a.chunk_row[ch0 + ch];
                    tc::mbar_arrive_expect_tx(&a_full[st], kGtStageBytes);
#pragma unroll
                    for (int hm = 0; hm < 2; ++hm) {
                        tc::tma_load_2d(sa + hm * kGtHalfBytes, &amap_re, t0b + 64 * hm, y, &a_full[st]);
                        tc::tma_load_2d(sa + hm * kGtHalfBytes + kGtHalfBytes / 2, &amap_im, t0b + 64 * hm, y,
                                        &a_full[st]);
                    }
                }
                if (!ok) break;
            }
            for (int gg = g - ns > 0 ? g - ns : 0; gg < g; ++gg)
                tc::mbar_wait_bounded(&a_full[gg % ns], (uint32_t)((gg / ns) & 1), kGtWaitCycles);
            tc::mbar_wait_bounded(b_full, 0, kGtWaitCycles);   // B has landed before the memory is released
        }
        __syncwarp();
    } else if (warp == kGtEpiWarps + 1) {
        // ---------------- MMA issuer (one lane)
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(128, NT, /*a_mn=*/true, /*b_mn=*/false);
            const uint32_t sb_sbo = (uint32_t)(kp / 8) * 128;
            const uint32_t sbb = tc::smem_u32(sB);
            int g = 0;
            bool ok = tc::mbar_wait_abortable(b_full, 0, kGtWaitCycles, abort_flag);
            for (int i = 0; i < nitems && ok; ++i) {
                const int b = i & 1;
                ok = tc::mbar_wait_abortable(&d_empty[b], (uint32_t)(((i >> 1) & 1) ^ 1), kGtWaitCycles, abort_flag);
                if (!ok) break;
                const uint32_t d = tbase + (uint32_t)(b * NT);
                for (int ch = 0; ch < nchunk; ++ch, ++g) {
                    const int st = g % ns;
                    ok = tc::mbar_wait_abortable(&a_full[st], (uint32_t)((g / ns) & 1), kGtWaitCycles,
                                                 abort_flag);
                    if (!ok) break;
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_u32(sA + st * kGtStageBytes);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        // k-step 0: the chunk's 16 real rows, 1: its 16 imaginary rows
                        const uint64_t ad = tc::smem_desc_sw128(sa + ks * 16 * 128, kGtHalfBytes, 1024);
                        const uint64_t bd = tc::smem_desc(sbb + (ch * (kGtChunkK / 8) + 2 * ks) * 128, 128, sb_sbo);
                        tc::mma_f16(d, ad, bd, idesc, ch > 0 || ks > 0);
                    }
                    tc::mma_commit(&a_empty[st]);
                }
                if (ok) tc::mma_commit(&d_full[b]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps 0-7: TMEM lanes 32 (w % 4) .. + 31 = samples; warp w / 4
        // drains half of the columns.  Column n = ((p 8 + cy) 2 + re/im) 8 + cx: every 8 columns are
        // one 16-byte piece (cy, re/im) of a sample's 256-byte row of the tile-major field
        // [channel][pol][tile row][tile col][sample][cy][re/im][cx]; 8 pieces of 32 samples make one
        // box (32 rows x 128 bytes, 128-byte swizzle) that one lane hands to the TMA unit.
        const int q4 = warp & 3, hc = warp >> 2;
        const int nty = a.N >> 3;
        unsigned char *boxes = sE + warp * a.boxes * kGtBoxBytes;
        int nbox = 0;
        for (int i = 0; i < nitems; ++i) {
            const int b = i & 1;
            if (!tc::mbar_wait_abortable(&d_full[b], (uint32_t)((i >> 1) & 1), kGtWaitCycles, abort_flag)) break;
            tc::fence_after_sync();
            const int cl = cb + i / ntb, t0w = (i % ntb) * 128 + q4 * 32;
            const uint32_t dcol = tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * NT);
            constexpr int NBX = NT / 2 / 64;              // boxes (64 columns each) per warp
#pragma unroll 1
            for (int bx = 0; bx < NBX; ++bx) {
                const int c0 = hc * (NT / 2) + 64 * bx;   // first column: piece c0 / 8
                float v[32], w[32];
                tc::tmem_ld32(dcol + (uint32_t)c0, v);
                tc::tmem_ld32(dcol + (uint32_t)(c0 + 32), w);
                if (bx == NBX - 1) {                      // the item's last TMEM read: the accumulator is free
                    tc::fence_before_sync();
                    tc::mbar_arrive(&d_empty[b]);
                }
                uint4 pk[8];
#pragma unroll
                for (int pc = 0; pc < 8; ++pc) {
                    const float *x = pc < 4 ? v + 8 * pc : w + 8 * (pc - 4);
                    __half2 h[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) h[u] = __floats2half2_rn(x[2 * u], x[2 * u + 1]);
                    pk[pc] = *reinterpret_cast<const uint4 *>(h);
                }
                unsigned char *box = boxes + (nbox % a.boxes) * kGtBoxBytes;
                if (nbox >= a.boxes) {                    // the store that last read this box is done with it
                    if (lane == 0) {
                        if (a.boxes == 2) tc::bulk_wait_read<1>();
                        else tc::bulk_wait_read<0>();
                    }
                    __syncwarp();
                }
#pragma unroll
                for (int pc = 0; pc < 8; ++pc)
                    *reinterpret_cast<uint4 *>(box + lane * 128 + ((pc ^ (lane & 7)) << 4)) = pk[pc];
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    const int grp0 = c0 >> 3, p = grp0 >> 4;   // 16 pieces per pol
                    const long long row = (((long long)(cl * P + p) * nty + ty) * nty + tx) * a.Tb + t0w;
                    tc::tma_store_2d(&gmap, tc::smem_u32(box), (grp0 & 15) * 8, (int)row);
                    tc::bulk_commit();
                }
                ++nbox;
            }
        }
        if (lane == 0) tc::bulk_wait_all();
    }
    if (*abort_flag && tid == 0) atomicExch(a.err, tc::kErrWaitTimeout);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, 2 * NT);
}

inline void tap_value(bool jones, int P, int K, const float *taps, int a, int po, int pi, int iy, int ix, float *re,
                      float *im) {
    long long idx;
    if (jones) {
        idx = ((((long long)a * 2 + po) * 2 + pi) * K + iy) * K + ix;
    } else {
        if (po != pi) { *re = 0.f; *im = 0.f; return; }
        idx = (((long long)a * P + po) * K + iy) * K + ix;
    }
    *re = taps[2 * idx];
    *im = taps[2 * idx + 1];
}

size_t kmajor_byte(int n, int k, int K) {
    return (size_t)(n >> 3) * (K >> 3) * 128 + (size_t)(k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

}  // namespace

size_t gridtc_smem_bytes(int P, int kp_max, int stages, int boxes) {
    const int NT = 128 * P;
    return 1024 + (((size_t)NT * kp_max * 2 + 1023) & ~(size_t)1023) + (size_t)stages * kGtStageBytes +
           (size_t)kGtEpiWarps * boxes * kGtBoxBytes + (size_t)(2 * stages + 5) * 8 + 16;
}

// A ring depth: the most stages (<= 8) that fit 227 KB beside B and the epilogue boxes; 0 if not even 4 fit.
int gridtc_stages(int P, int kp_max, int boxes) {
    for (int s = kGtMaxStages; s >= 4; --s)
        if (gridtc_smem_bytes(P, kp_max, s, boxes) <= 227 * 1024) return s;
    return 0;
}

// Store map of the tile-major gridded field as rows of 128 halves (one sample of one (pol, tile)):
// box 64 halves x 32 rows, 128-byte swizzle.
cudaError_t encode_gridtc_store_map(CUtensorMap *map, void *G, long long rows) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const cuuint64_t dims[2] = {128, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {256};
    const cuuint32_t box[2] = {64, 32};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, G, dims, strides, box, estr,
                                                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                                    CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tile tables of an array (host side, FP64 values rounded once to FP16 after the scale).
moff_status build_gridtc(int A, int K, int N, int P, bool jones, const double *pos, const float *taps, float scale,
                         GridTc *gt) {
    const int h = K / 2, NT = 128 * P, nty = N / 8;
    const int pin_n = jones ? 2 : 1;
    std::vector<int> ax(A), ay(A);
    for (int a = 0; a < A; ++a) {
        const long long fx = (long long)std::floor(pos[2 * a] + 0.5), fy = (long long)std::floor(pos[2 * a + 1] + 0.5);
        ax[a] = (int)(((fx % N) + N) % N);
        ay[a] = (int)(((fy % N) + N) % N);
    }
    // Plane rows: per anchor row (ascending), its antennas by anchor column, then again the
    // antennas whose column is below the window width (8 + 2h): a window that wraps the grid's
    // right edge continues into those copies, so every tile reads one run per anchor row.
    const int wlen = std::min(8 + 2 * h, N);
    std::vector<std::vector<int>> row_ant(N);
    for (int a = 0; a < A; ++a) row_ant[ay[a]].push_back(a);
    std::vector<int> row_first(N, 0), row_main(N, 0);   // first plane antenna slot of each row, its antenna count
    std::vector<int> slot_ant;                           // plane antenna slot -> antenna
    for (int yy = 0; yy < N; ++yy) {
        auto &ra = row_ant[yy];
        std::stable_sort(ra.begin(), ra.end(), [&](int x, int y) { return ax[x] < ax[y]; });
        row_first[yy] = (int)slot_ant.size();
        row_main[yy] = (int)ra.size();
        slot_ant.insert(slot_ant.end(), ra.begin(), ra.end());
        if (wlen < N)
            for (int a : ra)
                if (ax[a] < wlen) slot_ant.push_back(a);
    }
    gt->n_rows = (int)slot_ant.size() * P;
    gt->perm.assign((size_t)gt->n_rows, 0);
    for (size_t i = 0; i < slot_ant.size(); ++i)
        for (int q = 0; q < P; ++q) gt->perm[i * P + q] = slot_ant[i] * P + q;
    gt->tile_cell.clear();
    gt->kp.clear();
    gt->chunk_off.assign(1, 0);
    gt->chunk_row.clear();
    gt->bimg_off.clear();
    gt->bimg.clear();
    gt->active.assign((size_t)nty * nty, 0);
    gt->kp_max = 0;
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < nty; ++tx) {
            // one run per anchor row in [8 ty - h, 8 ty + 7 + h] (cyclic): the antennas whose anchor
            // column lies in [8 tx - h, 8 tx + 7 + h] (cyclic), as consecutive plane antenna slots
            struct Run { int r0, n; };
            std::vector<Run> runs;
            const int x0 = ((8 * tx - h) % N + N) % N;
            const bool wraps = x0 + wlen > N;
            for (int dy = 0; dy < std::min(8 + 2 * h, N); ++dy) {
                const int yy = ((8 * ty - h + dy) % N + N) % N;
                const auto &ra = row_ant[yy];
                int first = -1, n = 0;
                for (int k = 0; k < (int)ra.size(); ++k)          // main slots with column >= x0 (and < x0 + wlen)
                    if (ax[ra[k]] >= x0 && ax[ra[k]] < x0 + wlen) {
                        if (first < 0) first = row_first[yy] + k;
                        ++n;
                    }
                if (wraps) {                                       // then the copies with column < x0 + wlen - N
                    int dup = 0;
                    for (int a : ra)
                        if (ax[a] < wlen) {
                            if (ax[a] < x0 + wlen - N) {
                                if (first < 0) first = row_first[yy] + row_main[yy] + dup;
                                ++n;
                            }
                            ++dup;
                        }
                }
                if (n) runs.push_back(Run{first, n});
            }
            if (runs.empty()) continue;
            // chunks of 16 plane rows over each run (P rows per antenna)
            struct Chunk { int v0, vend; };
            std::vector<Chunk> ch;
            for (const Run &r : runs)
                for (int v = r.r0 * P; v < (r.r0 + r.n) * P; v += kGtChunkRows)
                    ch.push_back(Chunk{v, std::min(v + kGtChunkRows, (r.r0 + r.n) * P)});
            const int kp = (int)ch.size() * kGtChunkK;
            gt->kp_max = std::max(gt->kp_max, kp);
            gt->tile_cell.push_back((ty << 16) | tx);
            gt->active[(size_t)ty * nty + tx] = 1;
            gt->kp.push_back(kp);
            for (const Chunk &c : ch) gt->chunk_row.push_back(c.v0);
            gt->chunk_off.push_back((int)gt->chunk_row.size());
            // B image [NT][kp] K-major: k = 32 chunk + 16 re/im + row in chunk; n = ((p 8 + cy) 2 + re/im) 8 + cx
            const size_t off = gt->bimg.size();
            gt->bimg_off.push_back((long long)(off * 2));
            gt->bimg.resize(off + (size_t)NT * kp, __float2half(0.f));
            __half *B = gt->bimg.data() + off;
            for (size_t c = 0; c < ch.size(); ++c)
                for (int v = ch[c].v0; v < ch[c].vend; ++v) {
                    const int r = v - ch[c].v0, i = v / P, q = v % P, an = slot_ant[i];
                    for (int po = 0; po < P; ++po) {
                        if (!jones && po != q) continue;
                        for (int cy = 0; cy < 8; ++cy) {
                            const int dy = ((8 * ty + cy - ay[an] + h) % N + N) % N;
                            if (dy >= K) continue;
                            for (int cx = 0; cx < 8; ++cx) {
                                const int dx = ((8 * tx + cx - ax[an] + h) % N + N) % N;
                                if (dx >= K) continue;
                                float tr, ti;
                                tap_value(jones, P, K, taps, an, po, q, dy, dx, &tr, &ti);
                                const double wr = (double)tr * scale, wi = (double)ti * scale;
                                const int nre = ((po * 8 + cy) * 2 + 0) * 8 + cx, nim = ((po * 8 + cy) * 2 + 1) * 8 + cx;
                                const int kre = (int)c * kGtChunkK + r, kim = kre + kGtChunkRows;
                                // G_re = sum w_re y_re - w_im y_im ; G_im = sum w_im y_re + w_re y_im
                                auto put = [&](int n, int k, double val) {
                                    const __half hv = __float2half_rn((float)val);
                                    std::memcpy(reinterpret_cast<unsigned char *>(B) + kmajor_byte(n, k, kp), &hv, 2);
                                };
                                put(nre, kre, wr);
                                put(nre, kim, -wi);
                                put(nim, kre, wi);
                                put(nim, kim, wr);
                            }
                        }
                    }
                }
            (void)pin_n;
        }
    return MOFF_OK;
}

cudaError_t launch_grid_tc(const GridTcArgs &a, const CUtensorMap &are, const CUtensorMap &aim, const CUtensorMap &gmap,
                           int n_tiles, int cgroups, size_t smem, cudaStream_t st) {
    auto k = a.P == 1 ? k_grid_tc<1> : k_grid_tc<2>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(n_tiles, cgroups), kGtThreads, smem, st>>>(a, are, aim, gmap);
    return cudaGetLastError();
}

}  // namespace moff
