// FP64 small dense path: one CTA per replica, one thread per degree of freedom, the
// whole run segment inside one launch (replicas are independent, paper's closing
// discussion on trivially parallel simulations, so CTAs never wait on each other).
//
// Per fused iteration (kick index kappa): F = -M q from the CTA's q in shared memory
// (Eq. 5), end of the current step (B, O, sample), start of the next (O, B, A)
// (Eq. 2 integrated by the cited velocity Verlet scheme), and the per-replica
// partial sums of x_i x_j over the tracked pairs (Eq. 6).  State planes are [R][Np]
// FP64; M is [N][Np] FP64.
#include <algorithm>

#include "fth_internal.h"
#include "gle_device.cuh"

namespace fth {

__device__ __forceinline__ double open_unit64(uint32_t x) {
    return (double)(((x >> 9) << 1) | 1u) * 5.9604644775390625e-8;
}

template <int NS>
__device__ __forceinline__ void gle_normals64(uint32_t kappa, uint32_t i, uint32_t r,
                                              uint32_t k0, uint32_t k1, double (&xi)[2 * NS]) {
    constexpr int kCalls = (2 * NS + 3) / 4;
#pragma unroll
    for (int k = 0; k < kCalls; ++k) {
        const uint4 x = philox4x32_10(make_uint4(kappa, i, r, (uint32_t)k), k0, k1);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double rho = sqrt(-2.0 * log(open_unit64(w[2 * h])));
            double sn, cs;
            sincospi(2.0 * open_unit64(w[2 * h + 1]), &sn, &cs);
            if (4 * k + 2 * h < 2 * NS) xi[4 * k + 2 * h] = rho * cs;
            if (4 * k + 2 * h + 1 < 2 * NS) xi[4 * k + 2 * h + 1] = rho * sn;
        }
    }
}

template <int NS>
__global__ void __launch_bounds__(1024)
fp64_dense_kernel(GleF64 g, int N, int Np, const double* __restrict__ M, double* __restrict__ q,
                  double* __restrict__ p, double* __restrict__ s, uint32_t kappa0, int iters,
                  int prologue, int observable, const int32_t* __restrict__ pairs, int npairs,
                  double* __restrict__ partial, int acc_from) {
    extern __shared__ double sh[];
    double* qs = sh;        // [Np]
    double* xs = sh + Np;   // [Np]
    const int r = blockIdx.x;
    const int i = threadIdx.x;
    const int R = gridDim.x;
    const int64_t base = (int64_t)r * Np;
    const int64_t plane = (int64_t)R * Np;
    double v[NS];
    double qi = 0.0;
    if (i < N) {
        qi = q[base + i];
        v[0] = p[base + i];
#pragma unroll
        for (int a = 1; a < NS; ++a) v[a] = s[(a - 1) * plane + base + i];
    }
    for (int k = i; k < Np; k += blockDim.x) qs[k] = (k < N) ? q[base + k] : 0.0;
    __syncthreads();
    double* acc = partial + (int64_t)r * npairs;
    for (int it = 0; it < iters; ++it) {
        const bool pro = prologue && it == 0;
        const uint32_t kappa = kappa0 + (uint32_t)it;
        double mq = 0.0;
        if (i < N) {
            const double* mi = M + (int64_t)i * Np;
            for (int k = 0; k < N; ++k) mq = fma(mi[k], qs[k], mq);
        }
        __syncthreads();   // all reads of qs done before it is overwritten
        if (i < N) {
            double xi[2 * NS];
            gle_normals64<NS>(kappa, (uint32_t)i, (uint32_t)r + g.roff, g.key0, g.key1, xi);
            if (!pro) {
                v[0] = fma(-g.hdt, mq, v[0]);
                o_half<NS, double>(v, g.T, g.S, xi);
                xs[i] = observable ? qi : v[0];
            }
            o_half<NS, double>(v, g.T, g.S, xi + NS);
            v[0] = fma(-g.hdt, mq, v[0]);
            qi = fma(g.dt, v[0], qi);
            qs[i] = qi;
        }
        __syncthreads();
        const int f = prologue ? it - 1 : it;   // index of this fused launch in the segment
        if (!pro && f >= acc_from) {
            for (int e = i; e < npairs; e += blockDim.x)
                acc[e] = fma(xs[pairs[2 * e]], xs[pairs[2 * e + 1]], acc[e]);
        }
        // xs is rewritten only after the next iteration's barrier
    }
    if (i < N) {
        q[base + i] = qi;
        p[base + i] = v[0];
#pragma unroll
        for (int a = 1; a < NS; ++a) s[(a - 1) * plane + base + i] = v[a];
    }
}

cudaError_t launch_fp64_dense(int ns, const GleF64& g, int64_t N, int64_t Np, int64_t R,
                              const double* M, double* q, double* p, double* s, uint32_t kappa0,
                              int64_t nsteps, int primed_in, int observable,
                              const int32_t* pairs, int64_t npairs, double* partial,
                              int64_t acc_from, cudaStream_t st) {
    const int prologue = primed_in ? 0 : 1;
    const int iters = (int)nsteps + prologue;
    if (iters <= 0) return cudaSuccess;
    const int threads = (int)std::max<int64_t>(32, ((N + 31) / 32) * 32);
    const size_t shmem = sizeof(double) * 2 * (size_t)Np;
    // kappa0 is the kick index of the first iteration (the prologue's when unprimed)
#define FTH_F64_CASE(NSV)                                                                   \
    case NSV:                                                                               \
        fp64_dense_kernel<NSV><<<(unsigned)R, threads, shmem, st>>>(                        \
            g, (int)N, (int)Np, M, q, p, s, kappa0, iters, prologue, observable, pairs,     \
            (int)npairs, partial, (int)acc_from);                                           \
        break;
    switch (ns) {
        FTH_F64_CASE(1)
        FTH_F64_CASE(2)
        FTH_F64_CASE(3)
        FTH_F64_CASE(4)
        FTH_F64_CASE(5)
        default: return cudaErrorInvalidValue;
    }
#undef FTH_F64_CASE
    return cudaGetLastError();
}

}  // namespace fth
