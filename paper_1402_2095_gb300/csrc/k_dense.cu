// Dense path kernels: FP32 FFMA force GEMM and the element-wise fused GLE step.
//
// State planes are [Np][Rp] FP32, replica fastest.  The force kernel writes
// MQ = M q (the force is -MQ, Eq. 5); the element-wise kernel then applies, per
// (i, r), the end of the current step (B(dt/2), O(dt/2), sample) and the start of
// the next one (O(dt/2), B(dt/2), A(dt)) of the GLE velocity Verlet scheme (Eq. 2).
#include <cuda_bf16.h>

#include "fth_internal.h"
#include "gle_device.cuh"

namespace fth {

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// -------------------------------------------------------------- element-wise step
// Block = 32 rows x 32 replicas: warp w takes rows i0 + 4w .. + 3, eight lanes per row with
// four consecutive replicas each, so every state-plane access of a warp is four whole
// 128-byte row segments.  The new positions go through shared memory so the force
// operand q^T[r][i] is written as 128-byte runs of i (one replica per warp row).
template <int NS>
__global__ void __launch_bounds__(256, 4)
dense_gle_kernel(GleF32 g, int N, int R, int Rp, float* __restrict__ MQ, int mq_planes,
                 float* __restrict__ q, float* __restrict__ p, float* __restrict__ s,
                 uint32_t kappa, int flags, int observable, float* __restrict__ ps,
                 int64_t ps_ld, int64_t slot_off, int op_kind, void* op_hi, void* op_lo,
                 int Np) {
    // programmatic dependent launch both ways: this grid may be resident before the force
    // GEMM it follows has finished, so it waits for it before touching memory; then it
    // lets the next force GEMM start its setup on SMs it leaves free (that kernel waits
    // for this grid before reading q)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ float tq[32][33];                 // [replica][row] of the block's tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * 32, rp = blockIdx.y * 32;
    const int k = warp * 4 + (lane >> 3);        // row within the tile
    const int i = i0 + k;
    const int c0 = (lane & 7) * 4;               // first replica within the tile
    const int r0 = rp + c0;
    float qn[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < N && r0 < Rp) {
        const int64_t plane = (int64_t)Np * Rp;
        const int64_t off = (int64_t)i * Rp + r0;
        // the force may arrive as partial sums over K (one plane per K share)
        float4 mq4 = *reinterpret_cast<const float4*>(MQ + off);
        for (int pl = 1; pl < mq_planes; ++pl) {
            const float4 x = *reinterpret_cast<const float4*>(MQ + pl * plane + off);
            mq4.x += x.x;
            mq4.y += x.y;
            mq4.z += x.z;
            mq4.w += x.w;
        }
        // the force adds into MQ: leave it zero for the next launch
        if (flags & kZeroMQ) *reinterpret_cast<float4*>(MQ + off) = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 q4 = *reinterpret_cast<const float4*>(q + off);
        float4 v4[NS];
        v4[0] = *reinterpret_cast<const float4*>(p + off);
#pragma unroll
        for (int a = 1; a < NS; ++a) v4[a] = *reinterpret_cast<const float4*>(s + (a - 1) * plane + off);

        const float* qa = reinterpret_cast<const float*>(&q4);
        float samp[4] = {0.f, 0.f, 0.f, 0.f};
        // replicas two at a time: one pair stream of normals serves both
        gle_quad<NS>(q4, v4, mq4, g, kappa, (uint32_t)i, r0, R, flags, observable, samp);
        *reinterpret_cast<float4*>(q + off) = q4;
        *reinterpret_cast<float4*>(p + off) = v4[0];
#pragma unroll
        for (int a = 1; a < NS; ++a) *reinterpret_cast<float4*>(s + (a - 1) * plane + off) = v4[a];
        if ((flags & kDoSample) && (flags & kSampleBf16)) {
            // BF16 stack of the tensor-core accumulation pass, rounded to nearest
            const __nv_bfloat162 s01 = __floats2bfloat162_rn(samp[0], samp[1]);
            const __nv_bfloat162 s23 = __floats2bfloat162_rn(samp[2], samp[3]);
            uint2 v;
            v.x = *reinterpret_cast<const uint32_t*>(&s01);
            v.y = *reinterpret_cast<const uint32_t*>(&s23);
            *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(ps) + (int64_t)i * ps_ld +
                                      slot_off + r0) = v;
        } else if (flags & kDoSample) {
            *reinterpret_cast<float4*>(ps + (int64_t)i * ps_ld + slot_off + r0) =
                make_float4(samp[0], samp[1], samp[2], samp[3]);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) qn[e] = qa[e];
    }
    if (op_kind == kOpNone) return;               // uniform over the grid
#pragma unroll
    for (int e = 0; e < 4; ++e) tq[c0 + e][k] = qn[e];
    __syncthreads();
    const int ii = i0 + lane;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int rl = warp * 4 + m;              // replica within the tile
        const int r = rp + rl;
        if (r >= Rp || ii >= N) continue;
        const float x = tq[rl][lane];
        if (op_kind == kOpTf32) {
            static_cast<float*>(op_hi)[(int64_t)r * Np + ii] = to_tf32(x);
        } else {
            const __nv_bfloat16 hb = __float2bfloat16_rn(x);
            static_cast<__nv_bfloat16*>(op_hi)[(int64_t)r * Np + ii] = hb;
            static_cast<__nv_bfloat16*>(op_lo)[(int64_t)r * Np + ii] =
                __float2bfloat16_rn(x - __bfloat162float(hb));
        }
    }
}

cudaError_t launch_dense_gle(int ns, const GleF32& g, int64_t N, int64_t R, int64_t Rp,
                             float* MQ, int mq_planes, float* q, float* p, float* s,
                             uint32_t kappa,
                             int flags, int observable, float* ps, int64_t ps_ld, int64_t slot,
                             int op_kind, void* op_hi, void* op_lo, int64_t Np,
                             cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((N + 31) / 32), (unsigned)((Rp + 31) / 32));
    cfg.blockDim = dim3(256, 1);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int64_t slot_off = slot * Rp;
#define FTH_DENSE_CASE(NSV)                                                                   \
    case NSV: {                                                                               \
        const cudaError_t e = cudaLaunchKernelEx(                                             \
            &cfg, dense_gle_kernel<NSV>, g, (int)N, (int)R, (int)Rp, MQ, mq_planes, q, p, s,  \
            kappa, flags, observable, ps, ps_ld, slot_off, op_kind, op_hi, op_lo, (int)Np);   \
        if (e != cudaSuccess) return e;                                                       \
        break;                                                                                \
    }
    switch (ns) {
        FTH_DENSE_CASE(1)
        FTH_DENSE_CASE(2)
        FTH_DENSE_CASE(3)
        FTH_DENSE_CASE(4)
        FTH_DENSE_CASE(5)
        default: return cudaErrorInvalidValue;
    }
#undef FTH_DENSE_CASE
    return cudaGetLastError();
}

// -------------------------------------------------------------- FP32 FFMA force GEMM
// MQ[i][r] = sum_k M[i][k] q[k][r]; M is [Np][ldm] zero padded (Np multiple of 128),
// q is [Np][Rp] with zero rows beyond N.  Tile 64 x 64, BK 16, 256 threads, 4 x 4
// outputs per thread, double-buffered shared memory.
constexpr int kSgBM = 64, kSgBN = 64, kSgBK = 16;

__global__ void __launch_bounds__(256)
sgemm_force_kernel(const float* __restrict__ M, int64_t ldm, const float* __restrict__ q,
                   int Rp, float* __restrict__ MQ, int N, int K) {
    __shared__ __align__(16) float As[2][kSgBK][kSgBM];
    __shared__ __align__(16) float Bs[2][kSgBK][kSgBN];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int row0 = blockIdx.x * kSgBM, col0 = blockIdx.y * kSgBN;
    // loader coordinates
    const int a_row = tid / 4, a_k = (tid % 4) * 4;
    const int b_k = tid / 16, b_col = (tid % 16) * 4;
    const bool b_ok = col0 + b_col < Rp;

    float acc[4][4] = {};
    auto load = [&](int buf, int k0) {
        const float4 a = *reinterpret_cast<const float4*>(M + (int64_t)(row0 + a_row) * ldm + k0 + a_k);
        As[buf][a_k + 0][a_row] = a.x;
        As[buf][a_k + 1][a_row] = a.y;
        As[buf][a_k + 2][a_row] = a.z;
        As[buf][a_k + 3][a_row] = a.w;
        float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b_ok) b = *reinterpret_cast<const float4*>(q + (int64_t)(k0 + b_k) * Rp + col0 + b_col);
        *reinterpret_cast<float4*>(&Bs[buf][b_k][b_col]) = b;
    };
    const int nk = K / kSgBK;
    load(0, 0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load(cur ^ 1, (kt + 1) * kSgBK);
#pragma unroll
        for (int kk = 0; kk < kSgBK; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
        }
        __syncthreads();
    }
    const int c = col0 + tx * 4;
    if (c >= Rp) return;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int r = row0 + ty * 4 + x;
        if (r < N)
            *reinterpret_cast<float4*>(MQ + (int64_t)r * Rp + c) =
                make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
    }
}

// Replica counts in whole 128-column tiles: tile 128 x 128, BK 8, 256 threads as 16 x 16,
// each thread 8 x 8 outputs at rows {4ty .. 4ty + 3, 64 + 4ty ..} and columns {4tx ..,
// 64 + 4tx ..}, so each of the four float4 shared-memory reads of a k step is contiguous
// across the warp (no bank conflicts) and a k step reads 16 floats per 64 FMAs.  The next
// k tile goes through registers while this one is multiplied (double-buffered shared
// memory).  K is split KS ways over blockIdx.z; share z writes plane z of MQ ([KS][Np][Rp],
// summed by the element-wise step), so an N = 4096, R = 256 force starts 256 CTAs, two per
// SM (184 µs against 214 µs with K split 2 and 336 µs with 64 x 64 tiles).
template <int KS>
__global__ void __launch_bounds__(256, 2)
sgemm128_force_kernel(const float* __restrict__ M, int64_t ldm, const float* __restrict__ q,
                      int Rp, float* __restrict__ MQ, int N, int K) {
    constexpr int BM = 128, BN = 128, BK = 8;
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN, kz = blockIdx.z;
    const int nkt = K / BK;
    const int kbeg = (nkt * kz / KS) * BK, kend = (nkt * (kz + 1) / KS) * BK;
    // loaders: A is 128 rows x 8 k (thread: row tid / 2, k (tid & 1) * 4), B is 8 k x 128
    // columns (thread: k tid / 32, columns (tid & 31) * 4)
    const int a_row = tid >> 1, a_k = (tid & 1) * 4;
    const int b_k = tid >> 5, b_col = (tid & 31) * 4;
    const float* ga = M + (int64_t)(row0 + a_row) * ldm + a_k;
    const float* gb = q + (int64_t)b_k * Rp + col0 + b_col;
    float acc[8][8] = {};
    float4 ra = *reinterpret_cast<const float4*>(ga + kbeg);
    float4 rb = *reinterpret_cast<const float4*>(gb + (int64_t)kbeg * Rp);
    auto stage = [&](int buf) {
        As[buf][a_k + 0][a_row] = ra.x;
        As[buf][a_k + 1][a_row] = ra.y;
        As[buf][a_k + 2][a_row] = ra.z;
        As[buf][a_k + 3][a_row] = ra.w;
        *reinterpret_cast<float4*>(&Bs[buf][b_k][b_col]) = rb;
    };
    stage(0);
    __syncthreads();
    int cur = 0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        const bool more = k0 + BK < kend;
        if (more) {
            ra = *reinterpret_cast<const float4*>(ga + k0 + BK);
            rb = *reinterpret_cast<const float4*>(gb + (int64_t)(k0 + BK) * Rp);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
        }
        if (more) stage(cur ^ 1);
        __syncthreads();
        cur ^= 1;
    }
    float* out = MQ + (int64_t)kz * K * Rp;          // plane kz (K = Np)
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const int r = row0 + (x < 4 ? ty * 4 + x : 64 + ty * 4 + x - 4);
        if (r >= N) continue;
        float* o = out + (int64_t)r * Rp + col0;
        *reinterpret_cast<float4*>(o + tx * 4) = make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
        *reinterpret_cast<float4*>(o + 64 + tx * 4) =
            make_float4(acc[x][4], acc[x][5], acc[x][6], acc[x][7]);
    }
}

int sgemm_force_planes(int64_t Rp) { return Rp % 128 == 0 ? 4 : 1; }

cudaError_t launch_sgemm_force(const float* M, int64_t ldm, const float* q, int64_t Rp,
                               float* MQ, int64_t N, cudaStream_t st) {
    const int64_t Np = ((N + 127) / 128) * 128;
    const int ks = sgemm_force_planes(Rp);
    if (ks > 1) {
        dim3 grid((unsigned)(Np / 128), (unsigned)(Rp / 128), (unsigned)ks);
        if (ks == 4)
            sgemm128_force_kernel<4><<<grid, 256, 0, st>>>(M, ldm, q, (int)Rp, MQ, (int)N, (int)Np);
        else
            sgemm128_force_kernel<2><<<grid, 256, 0, st>>>(M, ldm, q, (int)Rp, MQ, (int)N, (int)Np);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)(Np / kSgBM), (unsigned)((Rp + kSgBN - 1) / kSgBN));
    sgemm_force_kernel<<<grid, 256, 0, st>>>(M, ldm, q, (int)Rp, MQ, (int)N, (int)Np);
    return cudaGetLastError();
}

// -------------------------------------------------------------- conversions
__global__ void round_tf32_kernel(float* x, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        x[k] = to_tf32(x[k]);
}

__global__ void split_bf16_kernel(const float* x, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x[k]);
        hi[k] = h;
        lo[k] = __float2bfloat16_rn(x[k] - __bfloat162float(h));
    }
}

cudaError_t launch_round_tf32(float* x, int64_t n, cudaStream_t st) {
    round_tf32_kernel<<<1216, 256, 0, st>>>(x, n);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(const float* x, int64_t n, void* hi, void* lo, cudaStream_t st) {
    split_bf16_kernel<<<1216, 256, 0, st>>>(x, n, static_cast<__nv_bfloat16*>(hi),
                                            static_cast<__nv_bfloat16*>(lo));
    return cudaGetLastError();
}

}  // namespace fth
