// Problem pools, device side: many independent problems resident on one GPU, stepped
// together by work-list kernels whose every input comes from a device descriptor table,
// so a whole chunk of steps can run from one captured CUDA graph.
//
// Per pool step (one fused launch of every problem, paper Eq. 2 / Eq. 5 / Eq. 6):
//   pool_force_kernel   dense problems: MQ = M q over (problem, 128-row block) items, a
//                       persistent tcgen05 kernel (tensor memory double-buffered so the
//                       epilogue of one item overlaps the MMAs of the next).  M and the
//                       q^T operand are stored pre-swizzled in 128-byte K slices, so plain
//                       bulk copies land them in the SWIZZLE_128B layout the MMA reads;
//   pool_gle_kernel     dense problems: the element-wise fused GLE step;
//   pool_csr_kernel     CSR problems: fused SpMM + GLE step;
//   pool_accum_kernel   items of up to 256 tracked pairs: accumulate this sample; the
//                       last item of a problem advances its counters and flushes its
//                       completed blocks.
// A problem's first launch is its prologue (start half only), exactly as a standalone
// context; its noise (key = its seed) and arithmetic order do not depend on the other
// problems in the pool, so its results are identical alone and in any mix.
#include <cuda_bf16.h>

#include <algorithm>

#include "fth_internal.h"
#include "gle_device.cuh"
#include "pool_internal.h"
#include "tc_primitives.cuh"

namespace fth {
using namespace tc;

// ------------------------------------------------------------------ force work list
template <int KIND, int RN, int STAGES>
struct PoolCfg {
    static constexpr int kOps = KIND == 1 ? 1 : 2;
    static constexpr int kABytes = 128 * 128;          // 128 rows x one 128-byte K slice
    static constexpr int kBBytes = RN * 128;
    static constexpr int kStageBytes = kOps * (kABytes + kBBytes);
    static constexpr int kTmemCols = (2 * RN) < 32 ? 32 : 2 * RN;   // two accumulators
    static constexpr size_t kSmem = (size_t)STAGES * kStageBytes + 1024 + 8 * (2 * STAGES + 5) + 16;
};

// Warp roles: warp 0 lane 0 bulk copies, warp 1 lane 0 issues the MMAs, warps 2..5
// (one per TMEM lane quadrant) drain the accumulators.  Items c, c + G, c + 2G ...
template <int KIND, int RN, int STAGES>
__global__ void __launch_bounds__(192, 1)
pool_force_kernel(const PoolDesc* __restrict__ desc, const PoolForceItem* __restrict__ items,
                  int nitems, uint32_t* err) {
    using C = PoolCfg<KIND, RN, STAGES>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* stages = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(stages + STAGES * C::kStageBytes);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;     // [2] MMA -> epilogue
    uint64_t* tempty = tfull + 2;         // [2] epilogue -> MMA
    uint64_t* drain = tempty + 2;         // MMA completion after a timed-out wait
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 128);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);
    constexpr int KS = KIND == 1 ? 32 : 64;   // K elements per 128-byte slice

    if (warp == 0 && lane == 0) {
        // producer
        int c = 0;
        bool ok = true;
        for (int j = blockIdx.x; j < nitems && ok; j += gridDim.x) {
            const PoolForceItem it = items[j];
            const PoolDesc& d = desc[it.problem];
            const int nks = d.np / KS;              // K slices per row block in the layout
            const int nk = (d.n + KS - 1) / KS;     // those past n are all zero padding
            const int J = it.rb, nb = d.np >> 7;
            const bool sym = KIND == 2 && d.sym;
            for (int kb = 0; kb < nk && ok; ++kb, ++c) {
                const int st = c % STAGES;
                if (c >= STAGES) ok = mbar_wait(&empty[st], ((c / STAGES) + 1) & 1, err);
                if (!ok) break;
                uint8_t* base = stages + st * C::kStageBytes;
                mbar_expect_tx(&full[st], C::kStageBytes);
                // A slice: byte offset within a plane, and whether it is the mirror's
                // transpose (two 8 KiB sub-tiles) or a plain K-major slice (16 KiB)
                size_t a_off;
                bool mn = false;
                if (sym) {
                    const int cb = kb >> 1, h = kb & 1;
                    if (cb >= J) {
                        a_off = (size_t)(J * nb - J * (J - 1) / 2 + (cb - J)) * 32768 + h * 16384;
                    } else {
                        a_off = (size_t)(cb * nb - cb * (cb - 1) / 2 + (J - cb)) * 32768 + h * 8192;
                        mn = true;
                    }
                } else {
                    a_off = ((size_t)J * nks + kb) * C::kABytes;
                }
                const int nplanes = KIND == 2 ? 2 : 1;
                for (int pl = 0; pl < nplanes; ++pl) {
                    const uint8_t* a = (pl ? d.a_lo : d.a_hi) + a_off;
                    uint8_t* sa = base + pl * (C::kABytes + C::kBBytes);
                    if (mn) {
                        bulk_load(sa, a, 8192, &full[st]);
                        bulk_load(sa + 8192, a + 16384, 8192, &full[st]);
                    } else {
                        bulk_load(sa, a, C::kABytes, &full[st]);
                    }
                    bulk_load(sa + C::kABytes, (pl ? d.bt_lo : d.bt_hi) + (size_t)kb * C::kBBytes,
                              C::kBBytes, &full[st]);
                }
            }
        }
        if (!ok) {
            for (int k = c > STAGES ? c - STAGES : 0; k < c; ++k)
                mbar_wait(&full[k % STAGES], (k / STAGES) & 1, err);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = (1u << 4) | ((uint32_t)(KIND == 1 ? 2 : 1) << 7) |
                                   ((uint32_t)(KIND == 1 ? 2 : 1) << 10) |
                                   ((uint32_t)(RN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        int c = 0, u = 0;
        bool ok = true;
        for (int j = blockIdx.x; j < nitems && ok; j += gridDim.x, ++u) {
            const int a = u & 1;
            if (u >= 2) ok = mbar_wait(&tempty[a], ((u >> 1) - 1) & 1, err);
            if (!ok) break;
            fence_after_sync();
            const PoolForceItem it = items[j];
            const PoolDesc& d = desc[it.problem];
            const int nk = (d.n + KS - 1) / KS;     // K slices past n are all zero padding
            const bool sym = KIND == 2 && d.sym;
            const uint32_t acc_t = tmem + (uint32_t)(a * RN);
            for (int kb = 0; kb < nk; ++kb, ++c) {
                const int st = c % STAGES;
                if (!mbar_wait(&full[st], (c / STAGES) & 1, err)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const bool mn = sym && (kb >> 1) < it.rb;
                const uint32_t base = smem_u32(stages + st * C::kStageBytes);
                const uint32_t abase_lo = base + C::kABytes + C::kBBytes;
                // K-major A advances 32 bytes per MMA (16 BF16 / 8 TF32 of K within the
                // swizzled row); MN-major A advances two 8-row K groups (2048 bytes)
                const uint64_t ah = mn ? sw128_mn_desc(base, 8192) : sw128_desc(base);
                const uint64_t al = mn ? sw128_mn_desc(abase_lo, 8192) : sw128_desc(abase_lo);
                const uint64_t bh = sw128_desc(base + C::kABytes);
                const uint32_t id = mn ? (idesc | (1u << 15)) : idesc;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t adv_b = (uint64_t)((kk * 32) >> 4);
                    const uint64_t adv_a = mn ? (uint64_t)((kk * 2048) >> 4) : adv_b;
                    const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                    if (KIND == 1) {
                        umma<1>(acc_t, ah + adv_a, bh + adv_b, id, acc);
                    } else {
                        const uint64_t bl = sw128_desc(base + 2 * C::kABytes + C::kBBytes);
                        umma<2>(acc_t, al + adv_a, bh + adv_b, id, acc);
                        umma<2>(acc_t, ah + adv_a, bl + adv_b, id, 1u);
                        umma<2>(acc_t, ah + adv_a, bh + adv_b, id, 1u);
                    }
                }
                umma_commit(&empty[st]);
            }
            umma_commit(&tfull[a]);
        }
        if (!ok) {
            // let every MMA issued so far finish before the tensor memory is freed
            atomicOr(err, kErrTimeout);
            umma_commit(drain);
            mbar_wait(drain, 0, err);
        }
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31
        const int q = warp & 3;
        int u = 0;
        for (int j = blockIdx.x; j < nitems; j += gridDim.x, ++u) {
            const int a = u & 1;
            // warp-uniform: tcgen05.ld below is .sync.aligned
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[a], (u >> 1) & 1, err));
            fence_after_sync();
            const PoolForceItem it = items[j];
            const PoolDesc& d = desc[it.problem];
            const int row = it.rb * 128 + q * 32 + lane;
            float* dst = d.mq + (size_t)row * RN;
#pragma unroll 1
            for (int c16 = 0; c16 < RN / 16; ++c16) {
                float v[16];
                if (ok) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * RN + c16 * 16), v);
                if (ok && row < d.n) {
#pragma unroll
                    for (int jj = 0; jj < 16; jj += 4)
                        *reinterpret_cast<float4*>(dst + c16 * 16 + jj) =
                            make_float4(v[jj], v[jj + 1], v[jj + 2], v[jj + 3]);
                }
            }
            fence_before_sync();
            mbar_arrive(&tempty[a]);
            if (!ok) break;
        }
    }
    __syncwarp();
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(C::kTmemCols));
    }
}

template <int KIND, int RN, int STAGES>
cudaError_t launch_pool_force_t(const PoolDesc* desc, const PoolForceItem* items, int nitems,
                                int grid, uint32_t* err, cudaStream_t st) {
    using C = PoolCfg<KIND, RN, STAGES>;
    static_assert(C::kSmem <= 232448, "shared memory");
    auto kern = pool_force_kernel<KIND, RN, STAGES>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
    kern<<<grid, 192, C::kSmem, st>>>(desc, items, nitems, err);
    return cudaGetLastError();
}

// Stage counts: "deep" fills ~200 KB of shared memory (one CTA per SM), "shallow" fits
// two CTAs per SM.
template <int KIND, int RN>
struct PoolStages {
    static constexpr int kStage = PoolCfg<KIND, RN, 1>::kStageBytes;
    static constexpr int kDeep = (200 * 1024) / kStage < 8 ? (200 * 1024) / kStage : 8;
    static constexpr int kShallow = (100 * 1024) / kStage < 4 ? (100 * 1024) / kStage : 4;
};

template <int KIND, int RN>
cudaError_t pool_force_rn(int variant, const PoolDesc* desc, const PoolForceItem* items,
                          int nitems, int grid, uint32_t* err, cudaStream_t st) {
    using S = PoolStages<KIND, RN>;
    if (variant == 0 || S::kShallow < 2)
        return launch_pool_force_t<KIND, RN, S::kDeep>(desc, items, nitems, grid, err, st);
    return launch_pool_force_t<KIND, RN, (S::kShallow < 2 ? 2 : S::kShallow)>(desc, items, nitems,
                                                                              grid, err, st);
}

cudaError_t launch_pool_force(int kind, int rn, int variant, const PoolDesc* desc,
                              const PoolForceItem* items, int nitems, int grid, uint32_t* err,
                              cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
#define FTH_POOL_RN(KV, RV) \
    if (kind == KV && rn == RV) return pool_force_rn<KV, RV>(variant, desc, items, nitems, grid, err, st);
    FTH_POOL_RN(1, 32)
    FTH_POOL_RN(1, 64)
    FTH_POOL_RN(1, 128)
    FTH_POOL_RN(2, 32)
    FTH_POOL_RN(2, 64)
    FTH_POOL_RN(2, 128)
#undef FTH_POOL_RN
    return cudaErrorInvalidValue;
}

int pool_force_max_ctas_per_sm(int kind, int rn, int variant) {
    (void)kind;
    (void)rn;
    return variant == 0 ? 1 : 2;
}

// ------------------------------------------------------------------ element-wise dense step
// Warp tasks: task = (32-row item, sub-block of 4 rows).  In each 32-replica pass a
// row is covered by 32 / NE lanes of NE consecutive replicas each, so every state load
// and store of a warp is whole 128-byte row segments.
// Warps are independent (no block barrier): each stages its problem's GLE constants in
// its own shared-memory slot, and transposes its new positions through a 4 x 32 slot
// to write the next force operand, q^T in the pre-swizzled slice layout the force
// kernel copies (slice kb = i / KS of RN rows x 128 bytes, 16-byte chunk c of row r at
// position c ^ (r & 7)): lane r writes replica r's 4 rows (TF32: 16 bytes; BF16: 8
// bytes of hi and 8 of lo).
constexpr int kPoolMaxRN = 128;

__device__ __forceinline__ float to_tf32_pool(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Per-warp copy of a problem's fields; the GLE constants every problem of a launch
// shares come as the kernel parameter `gk` (constant bank), only the noise keys and
// the replica offset are per problem.
struct PoolGleShared {
    uint32_t rk[20];
    uint32_t roff;
    float* q;
    float* p;
    float* s;
    float* mq;
    float* x;
    uint8_t* bt_hi;
    uint8_t* bt_lo;
    int n, flags, observable, primed;
    uint32_t kappa;
};

template <int NE> struct VecF;
template <> struct VecF<1> { using T = float; };
template <> struct VecF<2> { using T = float2; };
template <> struct VecF<4> { using T = float4; };

// NE consecutive replicas r0 .. r0 + NE - 1 of row i.
template <int NS, int NE>
__device__ __forceinline__ void pool_gle_vec(const PoolGleShared& c, const GleF32& gk, int i,
                                             int r0, int RN, float (&qout)[NE]) {
    using V = typename VecF<NE>::T;
    const size_t plane = (size_t)c.n * RN;
    const size_t off = (size_t)i * RN + r0;
    const V mq4 = *reinterpret_cast<const V*>(c.mq + off);
    V q4 = *reinterpret_cast<const V*>(c.q + off);
    V v4[NS];
    v4[0] = *reinterpret_cast<const V*>(c.p + off);
#pragma unroll
    for (int a = 1; a < NS; ++a) v4[a] = *reinterpret_cast<const V*>(c.s + (a - 1) * plane + off);
    float* qa = reinterpret_cast<float*>(&q4);
    const float* mqa = reinterpret_cast<const float*>(&mq4);
    V sv;
    float* samp = reinterpret_cast<float*>(&sv);
    if constexpr (NE == 1) {
        float v[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) v[a] = reinterpret_cast<float*>(&v4[a])[0];
        float xi[NS + 1];
        gle_normals<NS>(c.kappa, (uint32_t)i, (uint32_t)r0 + c.roff, c.rk, xi);
        samp[0] = 0.f;
        gle_fused<NS>(qa[0], v, mqa[0], gk, xi, c.flags, c.observable, samp[0]);
#pragma unroll
        for (int a = 0; a < NS; ++a) reinterpret_cast<float*>(&v4[a])[0] = v[a];
        qout[0] = qa[0];
    } else {
        // replicas two at a time: one pair stream of normals serves both
#pragma unroll
        for (int e = 0; e < NE; e += 2) {
            float xa[NS + 1], xb[NS + 1];
            gle_normals_two<NS>(c.kappa, (uint32_t)i, (uint32_t)(r0 + e) + c.roff, c.rk, xa, xb);
            if ((c.flags & kDoEnd) && (c.flags & kDoStart)) {
                // steady state: both replicas in the lanes of packed FP32 instructions
                float2 zeta[NS + 1];
#pragma unroll
                for (int k = 0; k <= NS; ++k) zeta[k] = make_float2(xa[k], xb[k]);
                float2 v[NS];
#pragma unroll
                for (int a = 0; a < NS; ++a) v[a] = reinterpret_cast<float2*>(&v4[a])[e >> 1];
                float2 q = reinterpret_cast<float2*>(&q4)[e >> 1];
                float2 sm;
                gle_fused2<NS>(q, v, reinterpret_cast<const float2*>(&mq4)[e >> 1], gk, zeta,
                               c.observable, sm);
#pragma unroll
                for (int a = 0; a < NS; ++a) reinterpret_cast<float2*>(&v4[a])[e >> 1] = v[a];
                reinterpret_cast<float2*>(&q4)[e >> 1] = q;
                samp[e] = sm.x;
                samp[e + 1] = sm.y;
                qout[e] = q.x;
                qout[e + 1] = q.y;
                continue;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ee = e + h;
                float v[NS];
#pragma unroll
                for (int a = 0; a < NS; ++a) v[a] = reinterpret_cast<float*>(&v4[a])[ee];
                samp[ee] = 0.f;
                if (h == 0) gle_fused<NS>(qa[ee], v, mqa[ee], gk, xa, c.flags, c.observable, samp[ee]);
                else gle_fused<NS>(qa[ee], v, mqa[ee], gk, xb, c.flags, c.observable, samp[ee]);
#pragma unroll
                for (int a = 0; a < NS; ++a) reinterpret_cast<float*>(&v4[a])[ee] = v[a];
                qout[ee] = qa[ee];
            }
        }
    }
    *reinterpret_cast<V*>(c.q + off) = q4;
    *reinterpret_cast<V*>(c.p + off) = v4[0];
#pragma unroll
    for (int a = 1; a < NS; ++a) *reinterpret_cast<V*>(c.s + (a - 1) * plane + off) = v4[a];
    if (c.primed) *reinterpret_cast<V*>(c.x + off) = sv;
}

// NE replicas per lane, MINB CTAs of 256 per SM (the register budget).  One block per item,
// no persistent task loop: the loop's carried state cost registers, and at the same
// occupancy the non-persistent form is 16 % faster on the ragged512 pool.
template <int NE, int MINB, int NS>
__global__ void __launch_bounds__(256, MINB)
pool_gle_kernel(const PoolDesc* __restrict__ desc, const PoolRowItem* __restrict__ items,
                int nitems, int RN, int kind, const GleF32 gk) {
    // one block per item (32 rows of one problem): warp w takes rows row0 + 4w .. + 3
    constexpr int LPR = 32 / NE;          // lanes per row: NE replicas each, 32 per pass
    __shared__ PoolGleShared c;
    __shared__ __align__(16) float sq[8][4 * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* tq = sq[warp];
    const PoolRowItem it = items[blockIdx.x];
    if (warp == 0) {
        const PoolDesc& d = desc[it.problem];
        if (lane < 20) c.rk[lane] = d.g.rk[lane];
        if (lane == 0) {
            c.roff = d.g.roff;
            c.q = d.q[0];
            c.p = d.p;
            c.s = d.s;
            c.mq = d.mq;
            c.x = d.x;
            c.bt_hi = d.bt_hi;
            c.bt_lo = d.bt_lo;
            c.n = d.n;
            c.primed = d.primed;
            c.flags = d.primed ? (kDoEnd | kDoStart) : kDoStart;
            c.observable = d.observable;
            c.kappa = (uint32_t)(d.primed ? d.t + 1 : d.t);
        }
    }
    __syncthreads();
    {
        const int row = it.row0 + warp * 4;         // first of the warp's 4 rows
        for (int rp = 0; rp < RN; rp += 32) {
#pragma unroll
            for (int h = 0; h < 4 / NE; ++h) {
                const int k = h * NE + lane / LPR;     // row within the 4
                const int i = row + k;
                const int r0 = rp + (lane % LPR) * NE;
                float qn[NE];
#pragma unroll
                for (int e = 0; e < NE; ++e) qn[e] = 0.f;
                if (i < c.n) pool_gle_vec<NS, NE>(c, gk, i, r0, RN, qn);
#pragma unroll
                for (int e = 0; e < NE; ++e) tq[k * 32 + (lane % LPR) * NE + e] = qn[e];
            }
            __syncwarp();
            const int r = rp + lane;                // this lane's replica
            float v[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = tq[m * 32 + lane];
            __syncwarp();
            if (kind == 1) {
                const int chunk = (row & 31) >> 2;
                const size_t o = (size_t)(row >> 5) * RN * 128 + (size_t)r * 128 +
                                 (size_t)((chunk ^ (r & 7)) << 4);
                *reinterpret_cast<float4*>(c.bt_hi + o) =
                    make_float4(to_tf32_pool(v[0]), to_tf32_pool(v[1]), to_tf32_pool(v[2]),
                                to_tf32_pool(v[3]));
            } else {
                __align__(8) __nv_bfloat16 hv[4], lv[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    hv[m] = __float2bfloat16_rn(v[m]);
                    lv[m] = __float2bfloat16_rn(v[m] - __bfloat162float(hv[m]));
                }
                const int col = (row & 63) * 2;     // byte column in the 128-byte row
                const size_t o = (size_t)(row >> 6) * RN * 128 + (size_t)r * 128 +
                                 (size_t)((((col >> 4) ^ (r & 7)) << 4) | (col & 15));
                *reinterpret_cast<uint2*>(c.bt_hi + o) = *reinterpret_cast<const uint2*>(hv);
                *reinterpret_cast<uint2*>(c.bt_lo + o) = *reinterpret_cast<const uint2*>(lv);
            }
        }
    }
}

template <int NE, int MINB, int NS>
cudaError_t launch_pool_gle_t(const PoolDesc* desc, const PoolRowItem* items, int nitems, int RN,
                              int kind, const GleF32& gk, cudaStream_t st) {
    pool_gle_kernel<NE, MINB, NS><<<nitems, 256, 0, st>>>(desc, items, nitems, RN, kind, gk);
    return cudaGetLastError();
}

template <int NS>
cudaError_t launch_pool_gle_ns(int variant, const PoolDesc* desc, const PoolRowItem* items,
                               int nitems, int RN, int kind, const GleF32& gk, cudaStream_t st) {
    switch (variant) {
        case 0: return launch_pool_gle_t<4, 3, NS>(desc, items, nitems, RN, kind, gk, st);
        case 1: return launch_pool_gle_t<2, 4, NS>(desc, items, nitems, RN, kind, gk, st);
        case 2: return launch_pool_gle_t<1, 5, NS>(desc, items, nitems, RN, kind, gk, st);
        case 3: return launch_pool_gle_t<4, 4, NS>(desc, items, nitems, RN, kind, gk, st);
        default: return cudaErrorInvalidValue;
    }
}

// Variants (replicas per lane, CTAs per SM) <4,3>, <2,4>, <1,5>, <4,4> (the last with a
// few spilled registers): every variant runs the same arithmetic per element, so they give
// identical results and the pool may time them on real steps.
// One launch covers the problems that share the GLE constants `gk` (ns of them).
cudaError_t launch_pool_gle(int variant, const PoolDesc* desc, const PoolRowItem* items,
                            int nitems, int RN, int kind, int ns, const GleF32& gk,
                            cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    if (RN > kPoolMaxRN || (RN & 31)) return cudaErrorInvalidValue;
    switch (ns) {
        case 1: return launch_pool_gle_ns<1>(variant, desc, items, nitems, RN, kind, gk, st);
        case 2: return launch_pool_gle_ns<2>(variant, desc, items, nitems, RN, kind, gk, st);
        case 3: return launch_pool_gle_ns<3>(variant, desc, items, nitems, RN, kind, gk, st);
        case 4: return launch_pool_gle_ns<4>(variant, desc, items, nitems, RN, kind, gk, st);
        case 5: return launch_pool_gle_ns<5>(variant, desc, items, nitems, RN, kind, gk, st);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ CSR fused step
// Warp tasks as in the dense step: 4 rows x 32 replicas per pass, 8 lanes per row with 4
// replicas each, so the state rows and every neighbour row q[j][r0 .. r0+3] a row's
// lanes gather are whole 128-byte segments; the row's column indices and values are
// broadcast loads.  Positions ping-pong between q[cur] and q[cur ^ 1].  One block per item
// (no persistent task loop) fits 64 registers, so four blocks per SM: on a serving mix of
// lattices that is 16 % faster than a persistent grid at three blocks per SM (80 registers)
// and 23 % faster than at two (116): the gathers need the warps in flight.
struct PoolCsrShared {
    uint32_t rk[20];
    uint32_t roff;
    const float* qin;
    float* qout;
    float* p;
    float* s;
    float* x;
    const int32_t* rowptr;
    const int32_t* col;
    const float* val;
    int n, flags, observable, primed;
    uint32_t kappa;
};

template <int NS>
__device__ __forceinline__ void pool_csr_quad(const PoolCsrShared& c, const GleF32& gk, int i,
                                              int r0, int RN) {
    const size_t plane = (size_t)c.n * RN;
    const size_t off = (size_t)i * RN + r0;
    float4 mq4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e1 = c.rowptr[i + 1];
    for (int e = c.rowptr[i]; e < e1; ++e) {
        const float m = c.val[e];
        const float4 x = *reinterpret_cast<const float4*>(c.qin + (size_t)c.col[e] * RN + r0);
        mq4.x = fmaf(m, x.x, mq4.x);
        mq4.y = fmaf(m, x.y, mq4.y);
        mq4.z = fmaf(m, x.z, mq4.z);
        mq4.w = fmaf(m, x.w, mq4.w);
    }
    float4 q4 = *reinterpret_cast<const float4*>(c.qin + off);
    float4 v4[NS];
    v4[0] = *reinterpret_cast<const float4*>(c.p + off);
#pragma unroll
    for (int a = 1; a < NS; ++a) v4[a] = *reinterpret_cast<const float4*>(c.s + (a - 1) * plane + off);
    float* qa = reinterpret_cast<float*>(&q4);
    const float* mqa = reinterpret_cast<const float*>(&mq4);
    float samp[4] = {0.f, 0.f, 0.f, 0.f};
    // replicas two at a time: one pair stream of normals serves both
#pragma unroll
    for (int e = 0; e < 4; e += 2) {
        float xa[NS + 1], xb[NS + 1];
        gle_normals_two<NS>(c.kappa, (uint32_t)i, (uint32_t)(r0 + e) + c.roff, c.rk, xa, xb);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ee = e + h;
            float v[NS];
#pragma unroll
            for (int a = 0; a < NS; ++a) v[a] = reinterpret_cast<float*>(&v4[a])[ee];
            if (h == 0) gle_fused<NS>(qa[ee], v, mqa[ee], gk, xa, c.flags, c.observable, samp[ee]);
            else gle_fused<NS>(qa[ee], v, mqa[ee], gk, xb, c.flags, c.observable, samp[ee]);
#pragma unroll
            for (int a = 0; a < NS; ++a) reinterpret_cast<float*>(&v4[a])[ee] = v[a];
        }
    }
    *reinterpret_cast<float4*>(c.qout + off) = q4;
    *reinterpret_cast<float4*>(c.p + off) = v4[0];
#pragma unroll
    for (int a = 1; a < NS; ++a) *reinterpret_cast<float4*>(c.s + (a - 1) * plane + off) = v4[a];
    if (c.primed)
        *reinterpret_cast<float4*>(c.x + off) = make_float4(samp[0], samp[1], samp[2], samp[3]);
}

template <int NS>
__global__ void __launch_bounds__(256, 4)
pool_csr_kernel(const PoolDesc* __restrict__ desc, const PoolRowItem* __restrict__ items,
                int nitems, int RN, const GleF32 gk) {
    // one block per item (32 rows of one problem): warp w takes rows row0 + 4w .. + 3
    __shared__ PoolCsrShared c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PoolRowItem it = items[blockIdx.x];
    if (warp == 0) {
        const PoolDesc& d = desc[it.problem];
        if (lane < 20) c.rk[lane] = d.g.rk[lane];
        if (lane == 0) {
            c.roff = d.g.roff;
            c.qin = d.q[d.cur];
            c.qout = d.q[d.cur ^ 1];
            c.p = d.p;
            c.s = d.s;
            c.x = d.x;
            c.rowptr = d.rowptr;
            c.col = d.col;
            c.val = d.val;
            c.n = d.n;
            c.primed = d.primed;
            c.flags = d.primed ? (kDoEnd | kDoStart) : kDoStart;
            c.observable = d.observable;
            c.kappa = (uint32_t)(d.primed ? d.t + 1 : d.t);
        }
    }
    __syncthreads();
    const int i = it.row0 + warp * 4 + (lane >> 3);
    if (i >= c.n) return;
    for (int r0 = (lane & 7) * 4; r0 < RN; r0 += 32) pool_csr_quad<NS>(c, gk, i, r0, RN);
}

template <int NS>
cudaError_t launch_pool_csr_t(const PoolDesc* desc, const PoolRowItem* items, int nitems, int RN,
                              const GleF32& gk, cudaStream_t st) {
    pool_csr_kernel<NS><<<nitems, 256, 0, st>>>(desc, items, nitems, RN, gk);
    return cudaGetLastError();
}

cudaError_t launch_pool_csr(const PoolDesc* desc, const PoolRowItem* items, int nitems, int RN,
                            int ns, const GleF32& gk, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    switch (ns) {
        case 1: return launch_pool_csr_t<1>(desc, items, nitems, RN, gk, st);
        case 2: return launch_pool_csr_t<2>(desc, items, nitems, RN, gk, st);
        case 3: return launch_pool_csr_t<3>(desc, items, nitems, RN, gk, st);
        case 4: return launch_pool_csr_t<4>(desc, items, nitems, RN, gk, st);
        case 5: return launch_pool_csr_t<5>(desc, items, nitems, RN, gk, st);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ convergence
// One CTA per live problem: over its tracked pairs, the normwise relative error bar of
// the block average, sqrt(sum_e M2_e / (nb (nb - 1))) / sqrt(sum_e mean_e^2), and the
// number nb of complete blocks, written to out[2 slot], out[2 slot + 1].
__global__ void __launch_bounds__(256)
pool_progress_kernel(const PoolDesc* __restrict__ desc, const int* __restrict__ live, int nlive,
                     double* __restrict__ out) {
    __shared__ double red[2][8];
    for (int j = blockIdx.x; j < nlive; j += gridDim.x) {
        const int slot = live[j];
        const PoolDesc& d = desc[slot];
        const double nb = (double)d.nblocks;
        double s2 = 0.0, mm = 0.0;
        if (nb >= 2.0)
            for (int e = threadIdx.x; e < d.npairs; e += blockDim.x) {
                s2 += d.m2[e];
                mm += d.mean[e] * d.mean[e];
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            mm += __shfl_xor_sync(0xffffffffu, mm, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = s2;
            red[1][threadIdx.x >> 5] = mm;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < 8; ++w) {
                a += red[0][w];
                b += red[1][w];
            }
            out[2 * slot] = nb >= 2.0 && b > 0.0 ? sqrt(a / (nb * (nb - 1.0))) / sqrt(b) : NAN;
            out[2 * slot + 1] = nb;
        }
        __syncthreads();
    }
}

cudaError_t launch_pool_progress(const PoolDesc* desc, const int* live, int nlive, double* out,
                                 cudaStream_t st) {
    if (nlive <= 0) return cudaSuccess;
    pool_progress_kernel<<<std::min(nlive, 152 * 4), 256, 0, st>>>(desc, live, nlive, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ operand conversion
// Rows [r0, r0 + nr) of a dense matrix (row-major, n columns, FP32 or FP64 at `src`,
// whose row 0 is row r0) into the force operand layout.  TF32 (kind 1): element (i, k)
// at byte ((i / 128 * (np / 32) + k / 32) * 128 + i % 128) * 128 + swizzled column, x
// rounded to nearest (ties away) as the tensor core reads it.  BF16X3 (kind 2): the
// upper 128 x 128 blocks only (M is symmetric, Eq. 5), each as four 64 x 64 sub-tiles
// (see PoolDesc), hi = bf16(x) and lo = bf16(x - hi), round-to-nearest-even.  In every
// layout the 16-byte chunk c of a 128-byte row r sits at chunk position c ^ (r & 7).
__global__ void pool_convert_kernel(const void* __restrict__ src, int f64, int n, int np,
                                    int r0, int nr, int kind, uint8_t* __restrict__ a_hi,
                                    uint8_t* __restrict__ a_lo) {
    const int64_t total = (int64_t)nr * n;
    const int ks = kind == 1 ? 32 : 64, esz = kind == 1 ? 4 : 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r0 + e / n, k = e % n;
        const float x = f64 ? (float)static_cast<const double*>(src)[e]
                            : static_cast<const float*>(src)[e];
        size_t o;
        if (kind == 1) {
            const int64_t r = i & 127, col = (k % ks) * esz;
            o = (size_t)((((i >> 7) * (np / ks) + k / ks) * 128 + r) * 128 +
                         ((((col >> 4) ^ (r & 7)) << 4) | (col & 15)));
        } else {
            // upper blocks only; a lower block is never stored (the mirror serves it)
            const int64_t I = i >> 7, J = k >> 7, nb = np >> 7;
            if (I > J) continue;
            const int64_t r = i & 127, cc = k & 127;
            const int64_t rr = r & 63, col = (cc & 63) * 2;
            o = (size_t)((I * nb - I * (I - 1) / 2 + (J - I)) * 32768 +
                         ((cc >> 6) * 2 + (r >> 6)) * 8192 + rr * 128 +
                         ((((col >> 4) ^ (rr & 7)) << 4) | (col & 15)));
        }
        if (kind == 1) {
            *reinterpret_cast<float*>(a_hi + o) = to_tf32_pool(x);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            *reinterpret_cast<__nv_bfloat16*>(a_hi + o) = h;
            *reinterpret_cast<__nv_bfloat16*>(a_lo + o) = __float2bfloat16_rn(x - __bfloat162float(h));
        }
    }
}

cudaError_t launch_pool_convert(const void* src, int f64, int n, int np, int r0, int nr, int kind,
                                uint8_t* a_hi, uint8_t* a_lo, cudaStream_t st) {
    if (nr <= 0) return cudaSuccess;
    const int64_t total = (int64_t)nr * n;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
    pool_convert_kernel<<<grid, 256, 0, st>>>(src, f64, n, np, r0, nr, kind, a_hi, a_lo);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ accumulate, advance, flush
// Items of up to kPoolAccChunk tracked pairs.  RN / 4 lanes share a pair: each loads one
// 16-byte vector of the two sample rows, so a warp's loads are whole rows (coalesced)
// rather than 32 scattered rows; the group's dot products are summed by shuffles and
// added to the pair's block partial.  Four passes of the block have their loads in
// flight together.  The last item of a problem to finish (a counter in its
// descriptor, after a fence) advances the problem's counters and, at a block end,
// folds the block means into the FP64 Welford sums.  A prologue launch only marks the
// problem primed.
template <int RN>
__global__ void __launch_bounds__(256)
pool_accum_kernel(PoolDesc* __restrict__ desc, const PoolAccItem* __restrict__ items, int nitems,
                  uint32_t* err) {
    __shared__ int s_last, s_flush;
    __shared__ double s_nb;
    for (int j = blockIdx.x; j < nitems; j += gridDim.x) {
        const PoolAccItem it = items[j];
        PoolDesc& d = desc[it.problem];
        const bool take = d.primed && d.nsamp >= d.burnin;
        if (take) {
            constexpr int kLanes = RN / 4;          // lanes per pair
            constexpr int kGroups = 256 / kLanes;   // pairs per pass
            constexpr int kBatch = 4;               // passes with loads in flight together
            const int sub = (int)threadIdx.x % kLanes, grp = (int)threadIdx.x / kLanes;
            for (int base = it.e0; base < it.e1; base += kBatch * kGroups) {
                int ea[kBatch];
                float4 u[kBatch], v[kBatch];
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    ea[k] = base + k * kGroups + grp;
                    u[k] = v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ea[k] < it.e1) {
                        const int ia = d.pairs[2 * ea[k]], ib = d.pairs[2 * ea[k] + 1];
                        u[k] = reinterpret_cast<const float4*>(d.x + (size_t)ia * RN)[sub];
                        v[k] = reinterpret_cast<const float4*>(d.x + (size_t)ib * RN)[sub];
                    }
                }
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    float acc = u[k].x * v[k].x;
                    acc = fmaf(u[k].y, v[k].y, acc);
                    acc = fmaf(u[k].z, v[k].z, acc);
                    acc = fmaf(u[k].w, v[k].w, acc);
#pragma unroll
                    for (int o = kLanes / 2; o > 0; o >>= 1)
                        acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (sub == 0 && ea[k] < it.e1) d.partial[ea[k]] += acc;
                }
            }
        }
        // the barrier orders every thread's partial store before thread 0's gpu-scope
        // fence, which releases them all before the completion count (the pattern of a
        // grid-wide barrier)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(&d.done, 1) == it.nchunks - 1;
            s_flush = 0;
            if (s_last) {
                __threadfence();
                d.done = 0;
                if (!d.primed) {
                    d.primed = 1;
                } else {
                    d.t += 1;
                    d.nsamp += 1;
                    if (take) {
                        d.inblock += 1;
                        if (d.inblock == d.block) {
                            s_flush = 1;
                            s_nb = (double)(d.nblocks + 1);
                        }
                    }
                }
                if (d.kind == 1) d.cur ^= 1;
            }
        }
        __syncthreads();
        if (s_flush) {
            // partial sums of the other items: read past L1, they were written this launch
            const double inv = 1.0 / ((double)d.block * (double)RN);
            bool bad = false;
            for (int k = threadIdx.x; k < d.npairs; k += blockDim.x) {
                const double bm = (double)__ldcg(d.partial + k) * inv;
                bad |= !isfinite(bm);
                const double dl = bm - d.mean[k];
                const double mu = d.mean[k] + dl / s_nb;
                d.m2[k] += dl * (bm - mu);
                d.mean[k] = mu;
                d.partial[k] = 0.f;
            }
            if (bad) atomicOr(err, kErrNonFinite);
            __syncthreads();
            if (threadIdx.x == 0) {
                d.nblocks += 1;
                d.inblock = 0;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_pool_accum(PoolDesc* desc, const PoolAccItem* items, int nitems, int RN,
                              uint32_t* err, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const int grid = std::min(nitems, 152 * 8);
    switch (RN) {
        case 32: pool_accum_kernel<32><<<grid, 256, 0, st>>>(desc, items, nitems, err); break;
        case 64: pool_accum_kernel<64><<<grid, 256, 0, st>>>(desc, items, nitems, err); break;
        case 128: pool_accum_kernel<128><<<grid, 256, 0, st>>>(desc, items, nitems, err); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace fth
