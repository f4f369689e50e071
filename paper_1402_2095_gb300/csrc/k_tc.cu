// tcgen05 / TMA kernels for sm_103a: the dense force GEMM (MQ = M q, Eq. 5) and the
// all-elements accumulator (SYRK of staged samples, Eq. 6 estimator).
//
// Both are D[128 x BN] += A[128 x K] B[BN x K]^T with A and B K-major in global
// memory.  TMA copies 128-byte-wide K slices (SWIZZLE_128B) into a ring of shared
// memory stages; one thread issues tcgen05.mma (kind::tf32: K = 8 per instruction, or
// kind::f16 with BF16 operands: K = 16) accumulating in tensor memory (one FP32
// column per output column, one TMEM lane per output row); tcgen05.commit releases a
// stage back to the TMA thread and finally signals the epilogue, where each of the 4
// warps reads its 32 TMEM lanes with tcgen05.ld.
//
// Every mbarrier wait is bounded (1 s of %globaltimer): on expiry the thread sets
// kErrTimeout in the device error word, the roles stop issuing work, outstanding TMA
// loads are drained with a bounded wait, and the CTA frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>

#include "fth_internal.h"
#include "tc_primitives.cuh"

namespace fth {
namespace {

using namespace tc;

// ------------------------------------------------------------------ shared mainloop
// KIND 1: TF32, one A and one B operand.  KIND 2: split BF16, A = (hi, lo),
// B = (hi, lo), three products hi*hi + hi*lo + lo*hi per K slice.  KIND 3: one BF16 A
// and B operand (the accumulation pass over the BF16 sample stack).
template <int KIND, int BN>
struct TcCfg {
    static constexpr int kOps = KIND == 2 ? 2 : 1;               // operand planes
    static constexpr int kABytes = 128 * 128;                     // one 128-row x 128-B slice
    static constexpr int kBBytes = BN * 128;
    static constexpr int kStageBytes = kOps * (kABytes + kBBytes);
    static constexpr int kKPerSlice = KIND == 1 ? 32 : 64;       // elements per 128 B
    static constexpr int kMmaPerSlice = 4;                        // 32 bytes of K each
    static constexpr int kTmemCols = BN < 32 ? 32 : BN;
};

struct TcMaps {
    CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

// a_blocks > 0: A is the blocked 3-D map with a_blocks K slices per row block.
// stall_ns > 0 (test hook, fth_test_stall): the producer issues no copies and the
// main-loop waits give up after stall_ns, so the launch ends through its timeout path
// with nothing in flight; the drain and epilogue waits keep the full bound.
template <int KIND, int BN, int STAGES>
__device__ __forceinline__ void tc_mainloop(const TcMaps& maps, int a_row, int b_row,
                                            int nslices, uint8_t* stages, uint64_t* full,
                                            uint64_t* empty, uint64_t* done, uint32_t tmem,
                                            uint32_t* err, int slice0 = 0, int a_blocks = 0,
                                            bool dep_wait = false, uint64_t stall_ns = 0) {
    using C = TcCfg<KIND, BN>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t loop_ns = stall_ns ? stall_ns : kWaitNs;
    if (warp == 0 && lane == 0 && stall_ns) {
        if (dep_wait) {
            grid_dependency_wait();
            allow_dependent_launch();
        }
        // nothing issued: a wait for the first release of slot 0, which nothing
        // releases, runs out (as the MMA thread's wait for its first stage does)
        if (nslices > 0) mbar_wait(&empty[0], 0, err, loop_ns);
    } else if (warp == 0 && lane == 0) {
        // TMA producer.  With dep_wait (a programmatic dependent launch whose B operand
        // is written by the previous kernel) the A slices of the first ring fill, which
        // no earlier kernel writes, are issued before the grid dependency wait.
        int issued = 0;
        bool ok = true;
        const int early = dep_wait ? std::min(STAGES, nslices) : 0;
        for (int kb = 0; kb < early; ++kb) {
            uint8_t* base = stages + kb * C::kStageBytes;
            mbar_expect_tx(&full[kb], C::kStageBytes);
            const int x = (slice0 + kb) * C::kKPerSlice;
            const int blk = (a_row / 128) * a_blocks + slice0 + kb;
            if (a_blocks > 0) tma_load_3d(&maps.a_hi, &full[kb], base, 0, 0, blk);
            else tma_load_2d(&maps.a_hi, &full[kb], base, x, a_row);
            if (KIND == 2) {
                if (a_blocks > 0) tma_load_3d(&maps.a_lo, &full[kb], base + C::kABytes + C::kBBytes, 0, 0, blk);
                else tma_load_2d(&maps.a_lo, &full[kb], base + C::kABytes + C::kBBytes, x, a_row);
            }
        }
        if (dep_wait) {
            grid_dependency_wait();
            allow_dependent_launch();
        }
        for (int kb = 0; kb < nslices && ok; ++kb) {
            const int st = kb % STAGES;
            if (kb >= STAGES) ok = mbar_wait(&empty[st], ((kb / STAGES) + 1) & 1, err);
            if (!ok) break;
            uint8_t* base = stages + st * C::kStageBytes;
            const int x = (slice0 + kb) * C::kKPerSlice;
            if (kb >= early) {
                mbar_expect_tx(&full[st], C::kStageBytes);
                const int blk = (a_row / 128) * a_blocks + slice0 + kb;
                if (a_blocks > 0) tma_load_3d(&maps.a_hi, &full[st], base, 0, 0, blk);
                else tma_load_2d(&maps.a_hi, &full[st], base, x, a_row);
                if (KIND == 2) {
                    if (a_blocks > 0) tma_load_3d(&maps.a_lo, &full[st], base + C::kABytes + C::kBBytes, 0, 0, blk);
                    else tma_load_2d(&maps.a_lo, &full[st], base + C::kABytes + C::kBBytes, x, a_row);
                }
            }
            tma_load_2d(&maps.b_hi, &full[st], base + C::kABytes, x, b_row);
            if (KIND == 2) tma_load_2d(&maps.b_lo, &full[st], base + 2 * C::kABytes + C::kBBytes, x, b_row);
            ++issued;
        }
        if (!ok || *reinterpret_cast<volatile uint32_t*>(err) != 0) {
            // drain the copies still in flight before the CTA exits (bounded)
            for (int kb = std::max(0, issued - STAGES); kb < issued; ++kb)
                mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, err);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = make_idesc(KIND == 1 ? 2 : 1, BN);
        bool ok = true;
        for (int kb = 0; kb < nslices; ++kb) {
            const int st = kb % STAGES;
            if (!mbar_wait(&full[st], (kb / STAGES) & 1, err, loop_ns)) {
                ok = false;
                break;
            }
            fence_after_sync();
            const uint32_t base = smem_u32(stages + st * C::kStageBytes);
            const uint64_t ah = sw128_desc(base);
            const uint64_t bh = sw128_desc(base + C::kABytes);
#pragma unroll
            for (int kk = 0; kk < C::kMmaPerSlice; ++kk) {
                const uint64_t adv = (uint64_t)((kk * 32) >> 4);   // 32 bytes per MMA K step
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                if (KIND == 1) {
                    umma<1>(tmem, ah + adv, bh + adv, idesc, acc);
                } else if (KIND == 3) {
                    umma<2>(tmem, ah + adv, bh + adv, idesc, acc);
                } else {
                    const uint64_t al = sw128_desc(base + C::kABytes + C::kBBytes);
                    const uint64_t bl = sw128_desc(base + 2 * C::kABytes + C::kBBytes);
                    umma<2>(tmem, al + adv, bh + adv, idesc, acc);   // lo * hi
                    umma<2>(tmem, ah + adv, bl + adv, idesc, 1u);    // hi * lo
                    umma<2>(tmem, ah + adv, bh + adv, idesc, 1u);    // hi * hi
                }
            }
            umma_commit(&empty[st]);
        }
        // always signal: the commit also tracks completion of every MMA issued above,
        // so the epilogue never frees TMEM under an MMA still in flight
        umma_commit(done);
        if (!ok) atomicOr(err, kErrTimeout);
    }
    __syncwarp();
}

template <int KIND, int BN, int STAGES>
__device__ __forceinline__ bool tc_setup(uint8_t*& stages, uint64_t*& full, uint64_t*& empty,
                                         uint64_t*& done, uint32_t& tmem) {
    using C = TcCfg<KIND, BN>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    stages = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * C::kStageBytes);
    full = bars;
    empty = bars + STAGES;
    done = bars + 2 * STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(C::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    tmem = *reinterpret_cast<volatile uint32_t*>(tslot);
    return true;
}

template <int KIND, int BN>
__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
    using C = TcCfg<KIND, BN>;
    fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(C::kTmemCols));
    }
}

// ------------------------------------------------------------------ force GEMM
// grid (Np / 128, ceil(Rp / BN)); MQ[row][col] for row < N, col < Rp.
template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(128, 1)
tc_force_kernel(const __grid_constant__ TcMaps maps, float* __restrict__ MQ, int ldf, int N,
                int Rp, int nslices, uint32_t* err, uint64_t stall_ns) {
    uint8_t* stages;
    uint64_t *full, *empty, *done;
    uint32_t tmem;
    tc_setup<KIND, BN, STAGES>(stages, full, empty, done, tmem);
    const int row0 = blockIdx.x * 128, col0 = blockIdx.y * BN;
    tc_mainloop<KIND, BN, STAGES>(maps, row0, col0, nslices, stages, full, empty, done, tmem, err,
                                  0, nslices, false, stall_ns);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warp-uniform: tcgen05.ld is .sync.aligned
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, err) &&
                                                *reinterpret_cast<volatile uint32_t*>(err) == 0);
    fence_after_sync();
    if (ok) {
        const int row = row0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < BN / 16; ++c) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
            if (row < N) {
                float* dst = MQ + (int64_t)row * ldf + col0 + c * 16;
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    if (col0 + c * 16 + j + 4 <= Rp)
                        *reinterpret_cast<float4*>(dst + j) =
                            make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
        }
    }
    tc_teardown<KIND, BN>(tmem);
}

// ------------------------------------------------------------------ split-K force GEMM
// The replicas of one 128-row block fit one tile (BN >= Rp).  The K range is split over
// the KSPLIT CTAs of a (1, KSPLIT, 1) cluster; each accumulates its K share in TMEM,
// stages the 128 x BN partial in its (now idle) shared memory, and after a cluster
// barrier reduces one BN/KSPLIT-column quarter of the tile across the cluster through
// distributed shared memory and writes it.  A second cluster barrier keeps every
// partial alive until all peers have read it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ float4 ld_cluster_f4(uint32_t local_saddr, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_saddr), "r"(rank));
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(remote)
                 : "memory");
    return v;
}

template <int KIND, int BN, int STAGES, int KSPLIT>
__global__ void __launch_bounds__(128, 1)
tc_force_splitk_kernel(const __grid_constant__ TcMaps maps, float* __restrict__ MQ, int ldf,
                       int N, int Rp, int nslices_total, uint32_t* err, uint64_t stall_ns) {
    constexpr int LDS = BN + 4;                 // padded row of the staged partial
    static_assert(STAGES * TcCfg<KIND, BN>::kStageBytes >= 128 * LDS * 4, "stage space");
    if (threadIdx.x == 64) {
        prefetch_tensormap(&maps.a_hi);
        prefetch_tensormap(&maps.b_hi);
        if (KIND == 2) {
            prefetch_tensormap(&maps.a_lo);
            prefetch_tensormap(&maps.b_lo);
        }
    }
    uint8_t* stages;
    uint64_t *full, *empty, *done;
    uint32_t tmem;
    tc_setup<KIND, BN, STAGES>(stages, full, empty, done, tmem);
    // programmatic dependent launch: setup above overlaps the previous kernel's tail;
    // q^T and MQ are touched only after the wait (the producer waits inside the mainloop)
    if (threadIdx.x != 0) {
        grid_dependency_wait();
        allow_dependent_launch();   // the element-wise kernel waits for this grid's end
    }
    const int row0 = blockIdx.x * 128;
    const int kc = (int)cluster_rank();
    const int s0 = (nslices_total * kc) / KSPLIT;
    const int s1 = (nslices_total * (kc + 1)) / KSPLIT;
    tc_mainloop<KIND, BN, STAGES>(maps, row0, 0, s1 - s0, stages, full, empty, done, tmem, err,
                                  s0, nslices_total, true, stall_ns);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool ok = mbar_wait(done, 0, err) && *reinterpret_cast<volatile uint32_t*>(err) == 0;
    fence_after_sync();
    float* red = reinterpret_cast<float*>(stages);
    const int row = warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < BN / 16; ++c) {
        float v[16];
        if (s1 > s0) {
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
        float4* dst = reinterpret_cast<float4*>(red + row * LDS + c * 16);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
    cluster_sync_all();
    constexpr int QW = BN / KSPLIT;             // columns reduced by this CTA
    constexpr int Q4 = QW / 4;
    const uint32_t red_s = smem_u32(red);
    for (int f = threadIdx.x; f < 128 * Q4; f += 128) {
        const int r = f / Q4;
        const int col = kc * QW + 4 * (f % Q4);
        const uint32_t off = red_s + (uint32_t)((r * LDS + col) * 4);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int src = 0; src < KSPLIT; ++src) {
            const float4 x = ld_cluster_f4(off, (uint32_t)src);
            acc.x += x.x;
            acc.y += x.y;
            acc.z += x.z;
            acc.w += x.w;
        }
        if (ok && row0 + r < N && col + 4 <= Rp)
            *reinterpret_cast<float4*>(MQ + (int64_t)(row0 + r) * ldf + col) = acc;
    }
    cluster_sync_all();
    tc_teardown<KIND, BN>(tmem);
}

// ------------------------------------------------------------------ row-pair force GEMM
// TF32, Rp in (128, 256], Np a multiple of 256.  A CTA takes two neighbouring 128-row blocks
// (rows rb0 * 128 .. + 255) over one of KSPLIT K shares: every q^T slice it loads feeds
// both blocks' MMAs (two 128 x 256 TMEM accumulators, all 512 columns), so a CTA takes in a
// third fewer operand bytes per flop than with one row block -- the operand intake of the
// SMs, not DRAM or L2 bandwidth, is what bounds the one-block kernel.  The partial tiles
// are added into MQ in L2 by TMA tensor reduce-adds from shared memory (SWIZZLE_128B boxes
// of 128 rows x 32 columns); MQ is zero at every launch (the element-wise step that reads
// it writes zeros back).  The order of the KSPLIT additions into an element is not fixed,
// so MQ can differ in its last bits from run to run.
template <int STAGES, int KSPLIT>
__global__ void __launch_bounds__(128, 1)
tc_force_pair_kernel(const __grid_constant__ TcMaps maps, const __grid_constant__ CUtensorMap mq,
                     int Rp, int nslices_total, uint32_t* err, uint64_t stall_ns) {
    constexpr int kA = 128 * 128;               // one 128-row x 128-B slice of M
    constexpr int kB = 256 * 128;               // 256 replica rows x 128 B of q^T
    constexpr int kStage = 2 * kA + kB;         // 64 KiB
    constexpr int kBox = 128 * 128;             // staged box: 128 rows x 32 FP32 columns
    static_assert(STAGES * kStage >= 8 * kBox, "stage space for one staged tile");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* stages = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(stages + STAGES * kStage);
    uint64_t* empty = full + STAGES;
    uint64_t* done = full + 2 * STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(full + 2 * STAGES + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 64) {
        prefetch_tensormap(&maps.a_hi);
        prefetch_tensormap(&maps.b_hi);
        prefetch_tensormap(&mq);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int q = 0; q < STAGES; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);
    // programmatic dependent launch: the setup above overlaps the previous kernel's tail;
    // q^T and MQ are touched only after the wait (the producer waits below)
    if (threadIdx.x != 0) {
        grid_dependency_wait();
        allow_dependent_launch();   // the element-wise kernel waits for this grid's end
    }
    const int rb0 = blockIdx.x * 2;             // first of the two 128-row blocks
    const int kc = blockIdx.y;
    const int s0 = (nslices_total * kc) / KSPLIT;
    const int nsl = (nslices_total * (kc + 1)) / KSPLIT - s0;
    const uint64_t loop_ns = stall_ns ? stall_ns : kWaitNs;

    if (warp == 0 && lane == 0) {
        // TMA producer
        if (stall_ns) {
            grid_dependency_wait();
            allow_dependent_launch();
            if (nsl > 0) mbar_wait(&empty[0], 0, err, loop_ns);
        } else {
            const int early = std::min(STAGES, nsl);
            // M slices of the first ring fill (no earlier kernel writes M) before the wait
            for (int kb = 0; kb < early; ++kb) {
                uint8_t* base = stages + kb * kStage;
                mbar_expect_tx(&full[kb], kStage);
                tma_load_3d(&maps.a_hi, &full[kb], base, 0, 0, rb0 * nslices_total + s0 + kb);
                tma_load_3d(&maps.a_hi, &full[kb], base + kA, 0, 0,
                            (rb0 + 1) * nslices_total + s0 + kb);
            }
            grid_dependency_wait();
            allow_dependent_launch();
            int issued = 0;
            bool ok = true;
            for (int kb = 0; kb < nsl && ok; ++kb) {
                const int st = kb % STAGES;
                if (kb >= STAGES) ok = mbar_wait(&empty[st], ((kb / STAGES) + 1) & 1, err);
                if (!ok) break;
                uint8_t* base = stages + st * kStage;
                if (kb >= early) {
                    mbar_expect_tx(&full[st], kStage);
                    tma_load_3d(&maps.a_hi, &full[st], base, 0, 0, rb0 * nslices_total + s0 + kb);
                    tma_load_3d(&maps.a_hi, &full[st], base + kA, 0, 0,
                                (rb0 + 1) * nslices_total + s0 + kb);
                }
                tma_load_2d(&maps.b_hi, &full[st], base + 2 * kA, (s0 + kb) * 32, 0);
                ++issued;
            }
            if (!ok || *reinterpret_cast<volatile uint32_t*>(err) != 0) {
                // drain the copies still in flight before the CTA exits (bounded)
                for (int kb = std::max(0, issued - STAGES); kb < issued; ++kb)
                    mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, err);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: block rb0 into TMEM columns 0..255, block rb0 + 1 into 256..511
        constexpr uint32_t idesc = make_idesc(2, 256);
        bool ok = true;
        for (int kb = 0; kb < nsl; ++kb) {
            const int st = kb % STAGES;
            if (!mbar_wait(&full[st], (kb / STAGES) & 1, err, loop_ns)) {
                ok = false;
                break;
            }
            fence_after_sync();
            const uint32_t base = smem_u32(stages + st * kStage);
            const uint64_t a0 = sw128_desc(base);
            const uint64_t a1 = sw128_desc(base + kA);
            const uint64_t b = sw128_desc(base + 2 * kA);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t adv = (uint64_t)((kk * 32) >> 4);   // 32 bytes per MMA K step
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                umma<1>(tmem, a0 + adv, b + adv, idesc, acc);
                umma<1>(tmem + 256u, a1 + adv, b + adv, idesc, acc);
            }
            umma_commit(&empty[st]);
        }
        // always signal: the commit also tracks completion of every MMA issued above
        umma_commit(done);
        if (!ok) atomicOr(err, kErrTimeout);
    }
    __syncwarp();

    // block-uniform: the staging loop below has block barriers
    const bool ok = __syncthreads_and(mbar_wait(done, 0, err) &&
                                      *reinterpret_cast<volatile uint32_t*>(err) == 0);
    fence_after_sync();                         // every stage consumed: reuse them for staging
    if (ok && nsl > 0) {
        // four chunks of 128 columns (two per tile), staged alternately in two 64 KiB
        // buffers: a chunk's reduce-adds run while the next chunk is read out of TMEM
        const int r = warp * 32 + lane;         // row within the 128-row block (TMEM lane)
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int t = q >> 1, half = q & 1;
            uint8_t* buf = stages + (q & 1) * 4 * kBox;
            if (q >= 2) {
                // the reduce-adds of chunk q - 2 have read this buffer
                if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                __syncthreads();
            }
#pragma unroll 1
            for (int g4 = 0; g4 < 2; ++g4) {
                uint32_t v[4][16];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    tmem_ld16_async(tmem + ((uint32_t)(warp * 32) << 16) +
                                        (uint32_t)(t * 256 + half * 128 + g4 * 64 + u * 16),
                                    v[u]);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    // columns 16 (4 g4 + u) .. + 15 of this chunk: box (2 g4 + u / 2), chunks
                    // (u & 1) * 4 .. + 3 of the row, each at j ^ (row mod 8) (SWIZZLE_128B)
                    uint8_t* box = buf + (2 * g4 + (u >> 1)) * kBox + r * 128;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int chunk = (u & 1) * 4 + j;
                        *reinterpret_cast<uint4*>(box + ((chunk ^ (r & 7)) << 4)) =
                            make_uint4(v[u][4 * j], v[u][4 * j + 1], v[u][4 * j + 2], v[u][4 * j + 3]);
                    }
                }
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int b = 0; b < 4; ++b) {
                    const int col = half * 128 + b * 32;
                    if (col < Rp) tma_reduce_add_2d(&mq, buf + b * kBox, col, (rb0 + t) * 128);
                }
                bulk_commit_group();
            }
        }
        if (threadIdx.x == 0) bulk_wait_all();
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ------------------------------------------------------------------ SYRK accumulator
// One CTA per upper tile (I <= J): tiles[t][a][b] += sum_c ps[I*128+a][c] ps[J*128+b][c].
template <int STAGES>
__global__ void __launch_bounds__(128, 1)
tc_syrk_kernel(const __grid_constant__ TcMaps maps, float* __restrict__ tiles, int nbt,
               int nslices, uint32_t* err) {
    uint8_t* stages;
    uint64_t *full, *empty, *done;
    uint32_t tmem;
    tc_setup<3, 128, STAGES>(stages, full, empty, done, tmem);
    int t = blockIdx.x, I = 0;
    while (t >= nbt - I) {
        t -= nbt - I;
        ++I;
    }
    const int J = I + t;
    tc_mainloop<3, 128, STAGES>(maps, I * 128, J * 128, nslices, stages, full, empty, done, tmem,
                                err);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warp-uniform: tcgen05.ld is .sync.aligned
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, err) &&
                                                *reinterpret_cast<volatile uint32_t*>(err) == 0);
    fence_after_sync();
    if (ok) {
        float* out = tiles + (int64_t)blockIdx.x * 128 * 128 + (int64_t)(warp * 32 + lane) * 128;
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
            float4* dst = reinterpret_cast<float4*>(out + c * 16);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float4 o = dst[j];
                o.x += v[4 * j];
                o.y += v[4 * j + 1];
                o.z += v[4 * j + 2];
                o.w += v[4 * j + 3];
                dst[j] = o;
            }
        }
    }
    tc_teardown<3, 128>(tmem);
}

// 128 x 256 tiles: rows I*128.., columns J'*256.. covering packed tiles (I, 2J') and
// (I, 2J'+1); only the tiles on or above the diagonal are accumulated.  Half the CTAs
// of the 128 x 128 form and 25 % fewer operand bytes per flop.
template <int STAGES>
__global__ void __launch_bounds__(128, 1)
tc_syrk_wide_kernel(const __grid_constant__ TcMaps maps, float* __restrict__ tiles, int nbt,
                    int nslices, uint32_t* err) {
    uint8_t* stages;
    uint64_t *full, *empty, *done;
    uint32_t tmem;
    tc_setup<3, 256, STAGES>(stages, full, empty, done, tmem);
    const int nbw = (nbt + 1) / 2;
    int t = blockIdx.x, I = 0;
    while (t >= nbw - I / 2) {
        t -= nbw - I / 2;
        ++I;
    }
    const int Jw = I / 2 + t;
    tc_mainloop<3, 256, STAGES>(maps, I * 128, Jw * 256, nslices, stages, full, empty, done, tmem,
                                err);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warp-uniform: tcgen05.ld is .sync.aligned
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, err) &&
                                                *reinterpret_cast<volatile uint32_t*>(err) == 0);
    fence_after_sync();
    if (ok) {
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const int J = 2 * Jw + half;
            if (J < I || J >= nbt) continue;
            const int64_t tile = (int64_t)I * nbt - ((int64_t)I * (I - 1)) / 2 + (J - I);
            float* out = tiles + tile * 128 * 128 + (int64_t)(warp * 32 + lane) * 128;
#pragma unroll 1
            for (int c = 0; c < 8; ++c) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(half * 128 + c * 16), v);
                float4* dst = reinterpret_cast<float4*>(out + c * 16);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float4 o = dst[j];
                    o.x += v[4 * j];
                    o.y += v[4 * j + 1];
                    o.z += v[4 * j + 2];
                    o.w += v[4 * j + 3];
                    dst[j] = o;
                }
            }
        }
    }
    tc_teardown<3, 256>(tmem);
}

// 256 x 256 output blocks (Iw <= Jw in 256-row units): two 128 x 256 accumulators (all
// 512 TMEM columns) share each B slice, so a CTA takes 64 KiB of operands per K slice for
// twice the MMAs of the 128 x 256 form (a third fewer operand bytes per flop).  On the
// diagonal A and B are the same rows and one load serves both.  Needs an even number of
// 128-row blocks.  BF16 operands (kind::f16, 64 K per 128-byte slice).  CTA c takes blocks
// c, c + G, c + 2G ... (G = min(blocks, SMs): one CTA fits an SM).  Warp 4 lane 0 issues the
// copies (running ahead into the next block
// while the accumulator drains), warp 5 lane 0 the MMAs, warps 0..3 (one TMEM lane
// quadrant each) drain the accumulator: 128-row x 32-column boxes staged in shared memory
// (SWIZZLE_128B, OUTB buffers) are added into the FP32 partial tiles in L2 by TMA tensor
// reduce-adds, so the read-modify-write of the partial sums never passes through the SM.
template <int STAGES, int OUTB>
__global__ void __launch_bounds__(192, 1)
tc_syrk_sq_kernel(const __grid_constant__ TcMaps maps, const __grid_constant__ CUtensorMap part,
                  int nbt, int nslices, uint32_t* err) {
    constexpr int kSlab = 256 * 128;            // one 256-row x 128-byte K slice
    constexpr int kStage = 2 * kSlab;           // A rows, then B rows
    constexpr int kBox = 128 * 128;             // staged box: 128 rows x 32 FP32 columns
    constexpr uint32_t kCols = 512;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* stages = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* stage_out = stages + STAGES * kStage;      // [OUTB][kBox]
    uint64_t* full = reinterpret_cast<uint64_t*>(stage_out + OUTB * kBox);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = full + 2 * STAGES;        // MMA -> epilogue
    uint64_t* tempty = tfull + 1;               // epilogue -> MMA
    uint64_t* drain = tfull + 2;                // MMA completion after a timed-out wait
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tfull + 3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 64) {
        prefetch_tensormap(&maps.a_hi);
        prefetch_tensormap(&maps.b_hi);
        prefetch_tensormap(&part);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, 128);
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);
    // programmatic dependent launch: the setup above overlaps the end of the element-wise
    // step that filled the stack; nothing of the stack or the partial tiles is touched
    // before that grid has finished, and the next force may set up during this pass
    grid_dependency_wait();
    allow_dependent_launch();
    const int nbw = nbt / 2;
    const int nblk = nbw * (nbw + 1) / 2;
    auto decode = [nbw](int t, int& Iw, int& Jw) {
        Iw = 0;
        while (t >= nbw - Iw) {
            t -= nbw - Iw;
            ++Iw;
        }
        Jw = Iw + t;
    };

    if (warp == 4 && lane == 0) {
        // TMA producer
        int c = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < nblk && ok; t += gridDim.x) {
            int Iw, Jw;
            decode(t, Iw, Jw);
            const bool diag = Iw == Jw;
            for (int kb = 0; kb < nslices; ++kb, ++c) {
                const int st = c % STAGES;
                if (c >= STAGES) ok = mbar_wait(&empty[st], ((c / STAGES) + 1) & 1, err);
                if (!ok) break;
                uint8_t* base = stages + st * kStage;
                mbar_expect_tx(&full[st], diag ? kSlab : kStage);
                tma_load_2d(&maps.b_hi, &full[st], base + kSlab, kb * 64, Jw * 256);
                if (!diag) tma_load_2d(&maps.b_hi, &full[st], base, kb * 64, Iw * 256);
            }
        }
        if (!ok || *reinterpret_cast<volatile uint32_t*>(err) != 0) {
            // drain the copies still in flight before the CTA exits (bounded)
            for (int k = c > STAGES ? c - STAGES : 0; k < c; ++k)
                mbar_wait(&full[k % STAGES], (k / STAGES) & 1, err);
        }
    } else if (warp == 5 && lane == 0) {
        // MMA issuer (BF16 operands): rows Iw*256 + 0..127 into columns 0..255, rows
        // + 128..255 into columns 256..511
        constexpr uint32_t idesc = make_idesc(1, 256);
        int c = 0, u = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < nblk && ok; t += gridDim.x, ++u) {
            int Iw, Jw;
            decode(t, Iw, Jw);
            const bool diag = Iw == Jw;
            // the previous block's accumulator has been read out
            if (u >= 1) ok = mbar_wait(tempty, (u - 1) & 1, err);
            if (!ok) break;
            fence_after_sync();
            for (int kb = 0; kb < nslices; ++kb, ++c) {
                const int st = c % STAGES;
                if (!mbar_wait(&full[st], (c / STAGES) & 1, err)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t base = smem_u32(stages + st * kStage);
                const uint32_t abase = diag ? base + kSlab : base;
                const uint64_t a0 = sw128_desc(abase);
                const uint64_t a1 = sw128_desc(abase + 128 * 128);
                const uint64_t b = sw128_desc(base + kSlab);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t adv = (uint64_t)((kk * 32) >> 4);
                    const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                    umma<2>(tmem, a0 + adv, b + adv, idesc, acc);
                    umma<2>(tmem + 256, a1 + adv, b + adv, idesc, acc);
                }
                umma_commit(&empty[st]);
            }
            if (ok) umma_commit(tfull);
        }
        if (!ok) {
            // let every MMA issued so far finish before the tensor memory is freed
            atomicOr(err, kErrTimeout);
            umma_commit(drain);
            mbar_wait(drain, 0, err);
        }
    } else if (warp < 4) {
        // epilogue: warp w reads TMEM lanes 32 w .. + 31 (rows of both 128-row halves)
        const int r = warp * 32 + lane;
        int u = 0, nbox = 0;
        for (int t = blockIdx.x; t < nblk; t += gridDim.x, ++u) {
            int Iw, Jw;
            decode(t, Iw, Jw);
            // uniform over the four warps: the box loop below has named barriers and
            // .sync.aligned TMEM loads
            const bool got = mbar_wait(tfull, u & 1, err);
            const bool ok = named_barrier_and(1, 128, got && *reinterpret_cast<volatile uint32_t*>(err) == 0);
            fence_after_sync();
            if (ok) {
#pragma unroll 1
                for (int q = 0; q < 16; ++q) {
                    // box q: accumulator columns 32 q .. + 31 = half-tile (a, half), box b
                    const int a = q >> 3, half = (q >> 2) & 1, b = q & 3;
                    const int I = 2 * Iw + a, J = 2 * Jw + half;
                    if (J < I) continue;                          // below the diagonal
                    uint8_t* buf = stage_out + (nbox % OUTB) * kBox;
                    if (nbox >= OUTB) {
                        // the reduce-add issued OUTB boxes ago has read this buffer
                        if (threadIdx.x == 0) {
                            if (OUTB == 2) bulk_wait_read_one();
                            else bulk_wait_read_all();
                        }
                        named_barrier(1, 128);
                    }
                    uint32_t v[2][16];
                    const uint32_t col = (uint32_t)(q * 32);
                    tmem_ld16_async(tmem + ((uint32_t)(warp * 32) << 16) + col, v[0]);
                    tmem_ld16_async(tmem + ((uint32_t)(warp * 32) << 16) + col + 16, v[1]);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<uint4*>(buf + r * 128 + ((j ^ (r & 7)) << 4)) =
                            make_uint4(v[j >> 2][4 * (j & 3)], v[j >> 2][4 * (j & 3) + 1],
                                       v[j >> 2][4 * (j & 3) + 2], v[j >> 2][4 * (j & 3) + 3]);
                    fence_proxy_async_smem();
                    named_barrier(1, 128);
                    if (threadIdx.x == 0) {
                        const int tile = I * nbt - (I * (I - 1)) / 2 + (J - I);
                        tma_reduce_add_3d(&part, buf, b * 32, 0, tile);
                        bulk_commit_group();
                    }
                    ++nbox;
                }
            }
            fence_before_sync();
            mbar_arrive(tempty);
            if (!ok) break;
        }
        // every reduce-add has landed before the block exits
        if (threadIdx.x == 0) bulk_wait_all();
    }
    __syncwarp();
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kCols));
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D K-major map: rows x cols elements, row stride ld elements, box (128 B) x box_rows.
cudaError_t make_map(CUtensorMap* map, const void* base, int bf16, uint64_t cols, uint64_t rows,
                     uint64_t ld, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const uint32_t esz = bf16 ? 2 : 4;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * esz};
    const cuuint32_t box[2] = {128u / esz, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 3-D map of M stored blocked: [Np/128][Np/KS][128][KS], KS = 128 bytes of K.
cudaError_t make_blocked_map(CUtensorMap* map, const void* base, int bf16, uint64_t Np) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const uint32_t esz = bf16 ? 2 : 4;
    const uint64_t ks = 128 / esz;
    const cuuint64_t dims[3] = {ks, 128, (Np / 128) * (Np / ks)};
    const cuuint64_t strides[2] = {ks * esz, 128 * ks * esz};
    const cuuint32_t box[3] = {(cuuint32_t)ks, 128, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kForceBN = 64;
constexpr int kForceStages = 6;
constexpr int kSyrkStages = 6;
constexpr int kSyrkWideStages = 4;
constexpr int kSyrkSqStages = 3;
constexpr int kSyrkOutBufs = 2;
constexpr int kWideBN = 256;
constexpr int kKSplit = 4;

template <int KIND, int BN, int STAGES>
size_t tc_smem_bytes() {
    return (size_t)STAGES * TcCfg<KIND, BN>::kStageBytes + 1024 + 8 * (2 * STAGES + 2);
}

}  // namespace

struct TcForce {
    CUtensorMap mq;     // MQ as 128-row x 32-column SWIZZLE_128B boxes (row-pair kernel)
    TcMaps maps;        // B box of kForceBN rows (column-tiled kernel)
    TcMaps maps_wide;   // B box of kWideBN rows (split-K kernel, Rp <= kWideBN)
    int kind;
    bool wide;
    bool pair;          // TF32 row-pair kernel with L2 reduce-adds (MQ zeroed by its reader)
    int64_t Np, Rp, N, R;
    uint64_t stall_ns = 0;   // test hook: > 0 makes the launches end through their timeout path
};

struct TcSyrk {
    TcMaps maps;        // A and B boxes of 128 rows
    TcMaps maps_wide;   // B box of 256 rows (Np >= 256)
    CUtensorMap part;   // FP32 partial tiles [ntiles][128][128], boxes of 128 x 32
    int64_t Np, ps_ld;
};

cudaError_t tc_force_prepare(TcForce** out, int kind, const void* A_hi, const void* A_lo,
                             const void* B_hi, const void* B_lo, int64_t Np, int64_t Rp,
                             int64_t N, int64_t R, float* MQ) {
    TcForce* tf = new TcForce();
    tf->kind = kind;
    tf->Np = Np;
    tf->Rp = Rp;
    tf->N = N;
    tf->R = R;
    const int bf = kind == 2;
    cudaError_t e = make_blocked_map(&tf->maps.a_hi, A_hi, bf, Np);
    if (e == cudaSuccess) e = make_map(&tf->maps.b_hi, B_hi, bf, Np, Rp, Np, kForceBN);
    if (e == cudaSuccess && bf) e = make_blocked_map(&tf->maps.a_lo, A_lo, bf, Np);
    if (e == cudaSuccess && bf) e = make_map(&tf->maps.b_lo, B_lo, bf, Np, Rp, Np, kForceBN);
    if (!bf) {
        tf->maps.a_lo = tf->maps.a_hi;
        tf->maps.b_lo = tf->maps.b_hi;
    }
    // replicas of a row block fit one 256-wide tile: split-K cluster kernel
    tf->wide = Rp > 128 && Rp <= kWideBN;
    if (e == cudaSuccess && tf->wide) {
        tf->maps_wide = tf->maps;
        e = make_map(&tf->maps_wide.b_hi, B_hi, bf, Np, Rp, Np, kWideBN);
        if (e == cudaSuccess && bf) e = make_map(&tf->maps_wide.b_lo, B_lo, bf, Np, Rp, Np, kWideBN);
        if (!bf) tf->maps_wide.b_lo = tf->maps_wide.b_hi;
    }
    // TF32 with whole pairs of row blocks: the row-pair kernel
    tf->pair = tf->wide && !bf && Np % 256 == 0 && MQ != nullptr;
    if (e == cudaSuccess && tf->pair) e = make_map(&tf->mq, MQ, 0, Rp, Np, Rp, 128);

    if (e != cudaSuccess) {
        delete tf;
        return e;
    }
    *out = tf;
    return cudaSuccess;
}

template <int KIND, int STAGES>
static cudaError_t launch_splitk(const TcForce* tf, float* MQ, int64_t ldf, uint32_t* err,
                                 cudaStream_t st) {
    const size_t sm = tc_smem_bytes<KIND, kWideBN, STAGES>();
    auto kern = tc_force_splitk_kernel<KIND, kWideBN, STAGES, kKSplit>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tf->Np / 128), kKSplit, 1);
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = kKSplit;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    const int nslices = (int)(KIND == 1 ? tf->Np / 32 : tf->Np / 64);
    return cudaLaunchKernelEx(&cfg, kern, tf->maps_wide, MQ, (int)ldf, (int)tf->N, (int)tf->Rp,
                              nslices, err, tf->stall_ns);
}


constexpr int kPairStages = 3;
constexpr int kPairKSplit = 9;

template <int KS>
static cudaError_t launch_pair_ks(const TcForce* tf, uint32_t* err, cudaStream_t st) {
    const size_t sm = (size_t)kPairStages * (2 * 128 * 128 + 256 * 128) + 1024 +
                      8 * (2 * kPairStages + 2);
    auto kern = tc_force_pair_kernel<kPairStages, KS>;
    static const bool attr_set =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
        cudaSuccess;
    (void)attr_set;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tf->Np / 256), KS, 1);
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, tf->maps_wide, tf->mq, (int)tf->Rp, (int)(tf->Np / 32),
                              err, tf->stall_ns);
}

// K split 9 fills 144 of the 152 SMs at N = 4096 (16 row pairs x 9; 8 ways left 24 idle);
// smaller problems split K 18 ways so they still start about as many CTAs (each CTA's
// partial tile, and so its epilogue, is the same size either way).
static cudaError_t launch_pair(const TcForce* tf, uint32_t* err, cudaStream_t st) {
    return tf->Np / 256 * kPairKSplit >= 96 ? launch_pair_ks<kPairKSplit>(tf, err, st)
                                            : launch_pair_ks<2 * kPairKSplit>(tf, err, st);
}

cudaError_t tc_force_run(const TcForce* tf, float* MQ, int64_t ldf, uint32_t* err,
                         cudaStream_t st) {
    if (tf->pair) {
        const cudaError_t e = launch_pair(tf, err, st);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    if (tf->wide) {
        cudaError_t e = tf->kind == 1 ? launch_splitk<1, 4>(tf, MQ, ldf, err, st)
                                      : launch_splitk<2, 2>(tf, MQ, ldf, err, st);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    dim3 grid((unsigned)(tf->Np / 128), (unsigned)((tf->Rp + kForceBN - 1) / kForceBN));
    if (tf->kind == 1) {
        constexpr int K = 1;
        const size_t sm = tc_smem_bytes<K, kForceBN, kForceStages>();
        auto kern = tc_force_kernel<K, kForceBN, kForceStages>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<grid, 128, sm, st>>>(tf->maps, MQ, (int)ldf, (int)tf->N, (int)tf->Rp,
                                    (int)(tf->Np / 32), err, tf->stall_ns);
    } else {
        constexpr int K = 2;
        constexpr int S = 4;
        const size_t sm = tc_smem_bytes<K, kForceBN, S>();
        auto kern = tc_force_kernel<K, kForceBN, S>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<grid, 128, sm, st>>>(tf->maps, MQ, (int)ldf, (int)tf->N, (int)tf->Rp,
                                    (int)(tf->Np / 64), err, tf->stall_ns);
    }
    return cudaGetLastError();
}

void tc_force_free(TcForce* tf) { delete tf; }

void tc_force_set_stall(TcForce* tf, uint64_t stall_ns) { tf->stall_ns = stall_ns; }

bool tc_force_accumulates(const TcForce* tf) { return tf->pair; }

cudaError_t tc_syrk_prepare(TcSyrk** out, const void* ps, int64_t Np, int64_t ps_ld,
                            float* tiles) {
    TcSyrk* ts = new TcSyrk();
    ts->Np = Np;
    ts->ps_ld = ps_ld;
    cudaError_t e = make_map(&ts->maps.a_hi, ps, 1, ps_ld, Np, ps_ld, 128);
    if (e != cudaSuccess) {
        delete ts;
        return e;
    }
    {
        const uint64_t nbt = (uint64_t)(Np / 128);
        const cuuint64_t dims[3] = {128, 128, nbt * (nbt + 1) / 2};
        const cuuint64_t strides[2] = {128 * 4, 128 * 128 * 4};
        const cuuint32_t box[3] = {32, 128, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        auto fn = encode_fn();
        if (!fn || fn(&ts->part, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, tiles, dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            delete ts;
            return fn ? cudaErrorInvalidValue : cudaErrorNotSupported;
        }
    }
    ts->maps.b_hi = ts->maps.a_hi;
    ts->maps.a_lo = ts->maps.a_hi;
    ts->maps.b_lo = ts->maps.a_hi;
    ts->maps_wide = ts->maps;
    if (Np >= 256) {
        e = make_map(&ts->maps_wide.b_hi, ps, 1, ps_ld, Np, ps_ld, 256);
        if (e != cudaSuccess) {
            delete ts;
            return e;
        }
    }
    *out = ts;
    return cudaSuccess;
}

cudaError_t tc_syrk_run(const TcSyrk* ts, int64_t ncols, float* tiles, uint32_t* err,
                        cudaStream_t st) {
    if (ncols <= 0) return cudaSuccess;
    const int nbt = (int)(ts->Np / 128);
    const int nslices = (int)((ncols + 63) / 64);   // BF16: 64 columns per 128-byte slice
    if (nbt >= 2 && nbt % 2 == 0) {
        const int nbw = nbt / 2;
        const int nblk = nbw * (nbw + 1) / 2;
        // one CTA per SM at most (shared memory): more blocks than SMs loop
        static const int nsm = [] {
            int dev = 0, n = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            return n > 0 ? n : 1;
        }();
        const unsigned grid = (unsigned)std::min(nblk, nsm);
        const size_t sm = (size_t)kSyrkSqStages * 2 * 256 * 128 + kSyrkOutBufs * 128 * 128 +
                          1024 + 8 * (2 * kSyrkSqStages + 4);
        auto kern = tc_syrk_sq_kernel<kSyrkSqStages, kSyrkOutBufs>;
        static const bool attr_set =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
            cudaSuccess;
        (void)attr_set;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid, 1, 1);
        cfg.blockDim = dim3(192, 1, 1);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e =
            cudaLaunchKernelEx(&cfg, kern, ts->maps_wide, ts->part, nbt, nslices, err);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    if (ts->Np >= 256) {
        const int nbw = (nbt + 1) / 2;
        unsigned nctas = 0;
        for (int I = 0; I < nbt; ++I) nctas += (unsigned)(nbw - I / 2);
        const size_t sm = tc_smem_bytes<3, 256, kSyrkWideStages>();
        auto kern = tc_syrk_wide_kernel<kSyrkWideStages>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<nctas, 128, sm, st>>>(ts->maps_wide, tiles, nbt, nslices, err);
        return cudaGetLastError();
    }
    const unsigned ntiles = (unsigned)(nbt * (nbt + 1) / 2);
    const size_t sm = tc_smem_bytes<3, 128, kSyrkStages>();
    auto kern = tc_syrk_kernel<kSyrkStages>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<ntiles, 128, sm, st>>>(ts->maps, tiles, nbt, nslices, err);
    return cudaGetLastError();
}

void tc_syrk_free(TcSyrk* ts) { delete ts; }

}  // namespace fth
