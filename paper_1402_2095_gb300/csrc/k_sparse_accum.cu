// Sparse path (fused CSR SpMM + GLE step) and the accumulation kernels.
//
// Sparse M (paper, Sec. "The f-thermostat": the force of Eq. 5 is a sparse
// matrix-vector product, O(N) per step): state planes are [N][Rp] FP32, replica
// fastest, so the gather of a neighbour row q[col][r..r+3] is one coalesced 16-byte
// vector per thread and the threads of a row read contiguous memory.
//
// Accumulation (Eq. 6 estimator, block averaging of the "2A" accumulators): samples
// are staged as ps[i][slot * Rp + r]; one pass adds sum_c ps[i][c] ps[j][c] over the
// staged columns to an FP32 block partial, and a block flush folds partial / (block R)
// into FP64 Welford (mean, M2) per element.
#include <algorithm>

#include "fth_internal.h"
#include "gle_device.cuh"

namespace fth {

// -------------------------------------------------------------- CSR fused step
// Thread t -> (row i = t / (Rp/4), replicas 4 * (t % (Rp/4)) .. +3).
template <int NS>
__global__ void __launch_bounds__(256, 4)
csr_step_kernel(GleF32 g, int N, int R, int Rp, const int32_t* __restrict__ rowptr,
                const int32_t* __restrict__ col, const float* __restrict__ val,
                const float* __restrict__ q_in, float* __restrict__ q_out,
                float* __restrict__ p, float* __restrict__ s, uint32_t kappa, int flags,
                int observable, float* __restrict__ ps, int64_t ps_ld, int64_t slot_off) {
    const int quads = Rp >> 2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * quads) return;
    const int i = (int)(t / quads);
    const int r0 = (int)(t % quads) * 4;
    const int64_t plane = (int64_t)N * Rp;
    const int64_t off = (int64_t)i * Rp + r0;

    float4 mq4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e1 = rowptr[i + 1];
    for (int e = rowptr[i]; e < e1; ++e) {
        const float m = val[e];
        const float4 x = *reinterpret_cast<const float4*>(q_in + (int64_t)col[e] * Rp + r0);
        mq4.x = fmaf(m, x.x, mq4.x);
        mq4.y = fmaf(m, x.y, mq4.y);
        mq4.z = fmaf(m, x.z, mq4.z);
        mq4.w = fmaf(m, x.w, mq4.w);
    }
    float4 q4 = *reinterpret_cast<const float4*>(q_in + off);
    float4 v4[NS];
    v4[0] = *reinterpret_cast<const float4*>(p + off);
#pragma unroll
    for (int a = 1; a < NS; ++a) v4[a] = *reinterpret_cast<const float4*>(s + (a - 1) * plane + off);

    float samp[4] = {0.f, 0.f, 0.f, 0.f};
    // replicas two at a time: one pair stream of normals serves both
    gle_quad<NS>(q4, v4, mq4, g, kappa, (uint32_t)i, r0, R, flags, observable, samp);
    *reinterpret_cast<float4*>(q_out + off) = q4;
    *reinterpret_cast<float4*>(p + off) = v4[0];
#pragma unroll
    for (int a = 1; a < NS; ++a) *reinterpret_cast<float4*>(s + (a - 1) * plane + off) = v4[a];
    if (flags & kDoSample)
        *reinterpret_cast<float4*>(ps + (int64_t)i * ps_ld + slot_off + r0) =
            make_float4(samp[0], samp[1], samp[2], samp[3]);
}

cudaError_t launch_csr_step(int ns, const GleF32& g, int64_t N, int64_t R, int64_t Rp,
                            const int32_t* rowptr, const int32_t* col, const float* val,
                            const float* q_in, float* q_out, float* p, float* s,
                            uint32_t kappa, int flags, int observable, float* ps,
                            int64_t ps_ld, int64_t slot, cudaStream_t st) {
    const int64_t threads = N * (Rp / 4);
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    const int64_t slot_off = slot * Rp;
#define FTH_CSR_CASE(NSV)                                                                      \
    case NSV:                                                                                  \
        csr_step_kernel<NSV><<<blocks, 256, 0, st>>>(g, (int)N, (int)R, (int)Rp, rowptr, col, val, \
                                                     q_in, q_out, p, s, kappa, flags,          \
                                                     observable, ps, ps_ld, slot_off);         \
        break;
    switch (ns) {
        FTH_CSR_CASE(1)
        FTH_CSR_CASE(2)
        FTH_CSR_CASE(3)
        FTH_CSR_CASE(4)
        FTH_CSR_CASE(5)
        default: return cudaErrorInvalidValue;
    }
#undef FTH_CSR_CASE
    return cudaGetLastError();
}

// -------------------------------------------------------------- pair accumulation
// One warp per tracked pair; ncols and ps_ld are multiples of 4.
__global__ void __launch_bounds__(256)
pair_accum_kernel(const float* __restrict__ ps, int64_t ps_ld, int64_t ncols,
                  const int32_t* __restrict__ pairs, int64_t npairs, float* __restrict__ partial) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= npairs) return;
    const float* a = ps + (int64_t)pairs[2 * w] * ps_ld;
    const float* b = ps + (int64_t)pairs[2 * w + 1] * ps_ld;
    float acc = 0.f;
    for (int64_t c = lane * 4; c < ncols; c += 128) {
        const float4 x = *reinterpret_cast<const float4*>(a + c);
        const float4 y = *reinterpret_cast<const float4*>(b + c);
        acc = fmaf(x.x, y.x, acc);
        acc = fmaf(x.y, y.y, acc);
        acc = fmaf(x.z, y.z, acc);
        acc = fmaf(x.w, y.w, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) partial[w] += acc;
}

cudaError_t launch_pair_accum(const float* ps, int64_t ps_ld, int64_t ncols,
                              const int32_t* pairs, int64_t npairs, float* partial,
                              cudaStream_t st) {
    if (npairs <= 0 || ncols <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((npairs * 32 + 255) / 256);
    pair_accum_kernel<<<blocks, 256, 0, st>>>(ps, ps_ld, ncols, pairs, npairs, partial);
    return cudaGetLastError();
}

// Row-grouped form: the tracked pairs sorted by their first index (CSR over rows:
// prow[i] .. prow[i+1] list the partners pcol and accumulator slots pe of row i).  A
// warp keeps row i of the staged samples in registers and streams its partners, so
// each row is read once for its own pairs instead of once per pair; for stencil-like
// pair lists (diagonal + lattice neighbours) the partner rows are near i and come
// from L2.  V float4 per lane: ncols = 128 V.
template <int V>
__global__ void __launch_bounds__(256)
pair_accum_rows_kernel(const float* __restrict__ ps, int64_t ps_ld, const int32_t* __restrict__ prow,
                       const int32_t* __restrict__ pcol, const int32_t* __restrict__ pe, int N,
                       float* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < N; i += nw) {
        const int k0 = prow[i], k1 = prow[i + 1];
        if (k0 == k1) continue;
        float4 a[V];
        const float4* ra = reinterpret_cast<const float4*>(ps + i * ps_ld);
#pragma unroll
        for (int v = 0; v < V; ++v) a[v] = ra[v * 32 + lane];
        // partners two at a time: both rows' loads are in flight before the FMAs
        for (int k = k0; k < k1; k += 2) {
            const bool two = k + 1 < k1;
            const float4* rb0 = reinterpret_cast<const float4*>(ps + (int64_t)pcol[k] * ps_ld);
            const float4* rb1 =
                reinterpret_cast<const float4*>(ps + (int64_t)pcol[two ? k + 1 : k] * ps_ld);
            float4 b0[V], b1[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                b0[v] = rb0[v * 32 + lane];
                b1[v] = rb1[v * 32 + lane];
            }
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                acc0 = fmaf(a[v].x, b0[v].x, acc0);
                acc1 = fmaf(a[v].x, b1[v].x, acc1);
                acc0 = fmaf(a[v].y, b0[v].y, acc0);
                acc1 = fmaf(a[v].y, b1[v].y, acc1);
                acc0 = fmaf(a[v].z, b0[v].z, acc0);
                acc1 = fmaf(a[v].z, b1[v].z, acc1);
                acc0 = fmaf(a[v].w, b0[v].w, acc0);
                acc1 = fmaf(a[v].w, b1[v].w, acc1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
                acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
            }
            if (lane == 0) {
                partial[pe[k]] += acc0;
                if (two) partial[pe[k + 1]] += acc1;
            }
        }
    }
}

bool pair_accum_rows_supported(int64_t ncols) {
    return ncols == 128 || ncols == 256 || ncols == 512 || ncols == 1024;
}

cudaError_t launch_pair_accum_rows(const float* ps, int64_t ps_ld, int64_t ncols,
                                   const int32_t* prow, const int32_t* pcol, const int32_t* pe,
                                   int64_t N, float* partial, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>((N * 32 + 255) / 256, 152 * 16);
    switch (ncols) {
        case 128: pair_accum_rows_kernel<1><<<blocks, 256, 0, st>>>(ps, ps_ld, prow, pcol, pe, (int)N, partial); break;
        case 256: pair_accum_rows_kernel<2><<<blocks, 256, 0, st>>>(ps, ps_ld, prow, pcol, pe, (int)N, partial); break;
        case 512: pair_accum_rows_kernel<4><<<blocks, 256, 0, st>>>(ps, ps_ld, prow, pcol, pe, (int)N, partial); break;
        case 1024: pair_accum_rows_kernel<8><<<blocks, 256, 0, st>>>(ps, ps_ld, prow, pcol, pe, (int)N, partial); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// -------------------------------------------------------------- FP32 FFMA SYRK
// tiles[t(I,J)][a][b] += sum_c ps[I*128+a][c] ps[J*128+b][c] for the upper tiles I <= J.
// 256 threads as 16 x 16, each 8 x 8 outputs at rows {4ty .. 4ty + 3, 64 + 4ty ..} and
// columns {4tx .., 64 + 4tx ..} (the four float4 shared-memory reads of a k step are
// contiguous across the warp: no bank conflicts); BK = 8; the next k tile goes through
// registers while this one is multiplied (double-buffered shared memory).
__global__ void __launch_bounds__(256, 2)
syrk_fp32_kernel(const float* __restrict__ ps, int64_t ps_ld, int64_t ncols, int nbt,
                 float* __restrict__ tiles) {
    constexpr int BK = 8;
    __shared__ __align__(16) float As[2][BK][kTile];
    __shared__ __align__(16) float Bs[2][BK][kTile];
    int t = blockIdx.x, I = 0;
    while (t >= nbt - I) {
        t -= nbt - I;
        ++I;
    }
    const int J = I + t;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int lr = tid >> 1, lk = (tid & 1) * 4;        // loader: row, first of 4 k
    const float* A = ps + ((int64_t)I * kTile + lr) * ps_ld + lk;
    const float* B = ps + ((int64_t)J * kTile + lr) * ps_ld + lk;
    float acc[8][8] = {};
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
    if (lk < ncols) {
        ra = *reinterpret_cast<const float4*>(A);
        rb = *reinterpret_cast<const float4*>(B);
    }
    auto stage = [&](int buf) {
        As[buf][lk + 0][lr] = ra.x;
        As[buf][lk + 1][lr] = ra.y;
        As[buf][lk + 2][lr] = ra.z;
        As[buf][lk + 3][lr] = ra.w;
        Bs[buf][lk + 0][lr] = rb.x;
        Bs[buf][lk + 1][lr] = rb.y;
        Bs[buf][lk + 2][lr] = rb.z;
        Bs[buf][lk + 3][lr] = rb.w;
    };
    stage(0);
    __syncthreads();
    int cur = 0;
    for (int64_t k0 = 0; k0 < ncols; k0 += BK) {
        const bool more = k0 + BK < ncols;
        if (more) {
            ra = rb = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k0 + BK + lk < ncols) {
                ra = *reinterpret_cast<const float4*>(A + k0 + BK);
                rb = *reinterpret_cast<const float4*>(B + k0 + BK);
            }
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
    float* out = tiles + (int64_t)blockIdx.x * kTile * kTile;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const int r = x < 4 ? ty * 4 + x : 64 + ty * 4 + x - 4;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4* o = reinterpret_cast<float4*>(out + r * kTile + h * 64 + tx * 4);
            float4 v = *o;
            v.x += acc[x][4 * h];
            v.y += acc[x][4 * h + 1];
            v.z += acc[x][4 * h + 2];
            v.w += acc[x][4 * h + 3];
            *o = v;
        }
    }
}

cudaError_t launch_syrk_fp32(const float* ps, int64_t ps_ld, int64_t ncols, int64_t Np,
                             float* tiles, cudaStream_t st) {
    const int nbt = (int)(Np / kTile);
    const unsigned ntiles = (unsigned)(nbt * (nbt + 1) / 2);
    syrk_fp32_kernel<<<ntiles, 256, 0, st>>>(ps, ps_ld, ncols, nbt, tiles);
    return cudaGetLastError();
}

// -------------------------------------------------------------- block flush
__global__ void flush_kernel(float* __restrict__ partial, double* __restrict__ mean,
                             double* __restrict__ m2, int64_t count, double inv_count, double nb,
                             uint32_t* err) {
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double b = (double)partial[e] * inv_count;
        bad |= !isfinite(b);
        const double d = b - mean[e];
        const double mu = mean[e] + d / nb;
        m2[e] += d * (b - mu);
        mean[e] = mu;
        partial[e] = 0.f;
    }
    if (bad) atomicOr(err, kErrNonFinite);
}

__global__ void flush64_kernel(double* __restrict__ partial, int64_t R, int64_t stride,
                               double* __restrict__ mean, double* __restrict__ m2, int64_t count,
                               double inv_count, double nb, uint32_t* err) {
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int64_t r = 0; r < R; ++r) {
            sum += partial[r * stride + e];
            partial[r * stride + e] = 0.0;
        }
        const double b = sum * inv_count;
        bad |= !isfinite(b);
        const double d = b - mean[e];
        const double mu = mean[e] + d / nb;
        m2[e] += d * (b - mu);
        mean[e] = mu;
    }
    if (bad) atomicOr(err, kErrNonFinite);
}

cudaError_t launch_flush(float* partial, double* mean, double* m2, int64_t count,
                         double inv_count, double nb, uint32_t* err, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>((count + 255) / 256, 152 * 16);
    flush_kernel<<<blocks, 256, 0, st>>>(partial, mean, m2, count, inv_count, nb, err);
    return cudaGetLastError();
}

cudaError_t launch_flush64(double* partial, int64_t R, int64_t stride, double* mean, double* m2,
                           int64_t count, double inv_count, double nb, uint32_t* err,
                           cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>((count + 255) / 256, 152 * 16);
    flush64_kernel<<<blocks, 256, 0, st>>>(partial, R, stride, mean, m2, count, inv_count, nb,
                                           err);
    return cudaGetLastError();
}

// -------------------------------------------------------------- linear functionals
// A functional L = sum_k w_k <x_{i_k} x_{j_k}> of tracked elements (e.g. Tr f(M) with
// unit weights on the diagonal, Tr O f(M) with the entries of a symmetric O, Eq. 6 and
// the trace forms of Sec. "The f-thermostat").  At each block flush, before the
// element partials are cleared, the block value sum_k w_k (block mean of element
// idx_k) is formed (acc[0], by atomics) and folded into FP64 Welford sums (acc[1],
// acc[2]) so the functional gets its own block error bar.
__global__ void functional_block_kernel(const float* __restrict__ partial32,
                                        const double* __restrict__ partial64, int64_t R,
                                        int64_t stride, const int64_t* __restrict__ idx,
                                        const double* __restrict__ w, int64_t nterms,
                                        double inv_count, double* __restrict__ acc) {
    double sum = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nterms;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = idx[k];
        double part = 0.0;
        if (partial32) part = (double)partial32[e];
        if (partial64)
            for (int64_t r = 0; r < R; ++r) part += partial64[r * stride + e];
        sum += w[k] * part * inv_count;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(acc, t);
    }
}

__global__ void functional_fold_kernel(double* __restrict__ acc, double nb, uint32_t* err) {
    const double b = acc[0];
    if (!isfinite(b)) atomicOr(err, kErrNonFinite);
    const double d = b - acc[1];
    const double mu = acc[1] + d / nb;
    acc[2] += d * (b - mu);
    acc[1] = mu;
    acc[0] = 0.0;
}

cudaError_t launch_functional_block(const float* partial32, const double* partial64, int64_t R,
                                    int64_t stride, const int64_t* idx, const double* w,
                                    int64_t nterms, double inv_count, double nb, double* acc,
                                    uint32_t* err, cudaStream_t st) {
    if (nterms > 0) {
        const unsigned blocks = (unsigned)std::min<int64_t>((nterms + 255) / 256, 152 * 4);
        functional_block_kernel<<<blocks, 256, 0, st>>>(partial32, partial64, R, stride, idx, w,
                                                        nterms, inv_count, acc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    functional_fold_kernel<<<1, 1, 0, st>>>(acc, nb, err);
    return cudaGetLastError();
}

// -------------------------------------------------------------- gather for fth_elements
__global__ void gather_kernel(const int64_t* __restrict__ idx, int64_t k,
                              const double* __restrict__ mean, const double* __restrict__ m2,
                              const float* __restrict__ partial32,
                              const double* __restrict__ partial64, int64_t p64_R,
                              int64_t p64_stride, double* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = idx[e];
        out[3 * e] = mean[x];
        out[3 * e + 1] = m2[x];
        double part = 0.0;
        if (partial32) part = (double)partial32[x];
        if (partial64)
            for (int64_t r = 0; r < p64_R; ++r) part += partial64[r * p64_stride + x];
        out[3 * e + 2] = part;
    }
}

cudaError_t launch_gather(const int64_t* idx, int64_t k, const double* mean, const double* m2,
                          const float* partial32, const double* partial64, int64_t p64_R,
                          int64_t p64_stride, double* out, cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>((k + 255) / 256, 1024);
    gather_kernel<<<blocks, 256, 0, st>>>(idx, k, mean, m2, partial32, partial64, p64_R,
                                          p64_stride, out);
    return cudaGetLastError();
}

}  // namespace fth
