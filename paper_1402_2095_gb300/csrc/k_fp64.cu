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

// Box-Muller in FP64 on one uint32 pair: rho = sqrt(-2 ln u_a), angle 2 pi u_b.
__device__ __forceinline__ void box_muller64(uint32_t a, uint32_t b, double& z0, double& z1) {
    const double rho = sqrt(-2.0 * log(open_unit64(a)));
    double sn, cs;
    sincospi(2.0 * open_unit64(b), &sn, &cs);
    z0 = rho * cs;
    z1 = rho * sn;
}

// Noise ahead of the integrator, already mixed by the O half-steps' noise factors: for
// every (kappa, i, r) of a segment of `iters` kick indices from kappa0 the kernel draws the
// W = NS + 1 normals zeta of the replica (replicas share streams in pairs, gle_device.cuh:
// global replica g = r + roff takes positions (g mod 2) W .. of the stream of pair g / 2)
// and writes c = L zeta, the noise terms of the two O half-steps drawn jointly (c_0 that of
// the sample, c_1..NS that of the next state), to xi[((it R + r) W + a) Np + i]; for the
// prologue's kick (pro0, it = 0) it writes c_1..NS = S zeta_0..NS-1 (one half-step), c_0 = 0.
// FP64 transcendental functions and these products are the bulk of the FP64 path's work;
// this kernel spreads them over the whole GPU while the integrator (one CTA per replica)
// keeps only the state-dependent arithmetic.  One thread per (it, pair, i), i fastest, so
// the stores coalesce.
template <int NS>
__global__ void __launch_bounds__(256)
fp64_noise_kernel(GleF64 g, int N, int Np, int R, uint32_t kappa0, int iters, int pro0,
                  double* __restrict__ xi) {
    constexpr int W = NS + 1;
    constexpr int kCalls = (2 * W + 3) / 4;
    const uint32_t j0 = g.roff >> 1;                         // first pair of this run
    const int npairs = (int)(((g.roff + (uint32_t)R - 1u) >> 1) - j0 + 1u);
    const int64_t total = (int64_t)iters * npairs * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % N);
        const int64_t rest = e / N;
        const uint32_t j = j0 + (uint32_t)(rest % npairs);
        const int it = (int)(rest / npairs);
        double z[4 * kCalls];                                // stream positions 0 .. 2W-1
#pragma unroll
        for (int k = 0; k < kCalls; ++k) {
            const uint4 x = philox4x32_10(make_uint4(kappa0 + (uint32_t)it, (uint32_t)i, j,
                                                     (uint32_t)k), g.key0, g.key1);
            box_muller64(x.x, x.y, z[4 * k], z[4 * k + 1]);
            if (4 * k + 2 < 2 * W) box_muller64(x.z, x.w, z[4 * k + 2], z[4 * k + 3]);
        }
        const bool pro = pro0 && it == 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = (int64_t)(2u * j + (uint32_t)h) - (int64_t)g.roff;   // local replica
            if (r < 0 || r >= R) continue;
            const double* zz = z + h * W;
            double* out = xi + ((int64_t)it * R + r) * W * Np + i;
            if (pro) {
                out[0] = 0.0;
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    double c = 0.0;
#pragma unroll
                    for (int b = 0; b <= a; ++b) c = fma(g.S[a * kMaxNs + b], zz[b], c);
                    out[(int64_t)(a + 1) * Np] = c;
                }
            } else {
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    double c = 0.0;
#pragma unroll
                    for (int b = 0; b <= a; ++b) c = fma(g.L[a * kMaxNs1 + b], zz[b], c);
                    out[(int64_t)a * Np] = c;
                }
            }
        }
    }
}

// O updates of the FP64 integrator with the noise terms c premixed by fp64_noise_kernel:
// v <- v + D v + c_1..NS (D = T - I for the prologue's half-step, T T - I for the joint
// pair), and the sample p = v_0 + (T v)_0 - v_0 + c_0 before it.
template <int NS>
__device__ __forceinline__ void o_apply64(double (&v)[NS], const double* D, const double* c) {
    double out[NS];
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        double acc = c[a + 1];
#pragma unroll
        for (int b = 0; b < NS; ++b) acc = fma(D[a * kMaxNs + b], v[b], acc);
        out[a] = v[a] + acc;
    }
#pragma unroll
    for (int a = 0; a < NS; ++a) v[a] = out[a];
}

template <int NS>
__device__ __forceinline__ double o_sample64(const double (&v)[NS], const GleF64& g,
                                             const double* c) {
    double inc = c[0];
#pragma unroll
    for (int b = 0; b < NS; ++b) inc = fma(g.T[b], v[b], inc);
    return v[0] + inc;
}

// Shared memory: q and the sample x ([Np] each); when they fit, M transposed
// ([N][Np], so a warp's row reads are conflict-free), the tracked pairs and their
// per-replica partial sums (written back at the end of the segment).
template <int NS>
__global__ void __launch_bounds__(1024)
fp64_dense_kernel(GleF64 g, int N, int Np, const double* __restrict__ M, double* __restrict__ q,
                  double* __restrict__ p, double* __restrict__ s, const double* __restrict__ noise,
                  int iters, int prologue, int observable, const int32_t* __restrict__ pairs,
                  int npairs, double* __restrict__ partial, int acc_from, int m_smem,
                  int p_smem) {
    extern __shared__ double sh[];
    double* qs = sh;                          // [Np]
    double* xs = sh + Np;                     // [Np]
    double* mt = xs + Np;                     // [N][Np] when m_smem
    double* pacc = mt + (m_smem ? (int64_t)N * Np : 0);             // [npairs] when p_smem
    int32_t* pidx = reinterpret_cast<int32_t*>(pacc + (p_smem ? npairs : 0));
    const int r = blockIdx.x;
    const int i = threadIdx.x;
    const int R = gridDim.x;
    const int64_t base = (int64_t)r * Np;
    const int64_t plane = (int64_t)R * Np;
    double* gacc = partial + (int64_t)r * npairs;
    double v[NS];
    double qi = 0.0;
    if (i < N) {
        qi = q[base + i];
        v[0] = p[base + i];
#pragma unroll
        for (int a = 1; a < NS; ++a) v[a] = s[(a - 1) * plane + base + i];
    }
    for (int k = i; k < Np; k += blockDim.x) qs[k] = (k < N) ? q[base + k] : 0.0;
    if (m_smem)
        for (int e = i; e < N * N; e += blockDim.x) {
            const int row = e / N, k = e % N;
            mt[(int64_t)k * Np + row] = M[(int64_t)row * Np + k];
        }
    if (p_smem)
        for (int e = i; e < npairs; e += blockDim.x) {
            pacc[e] = gacc[e];
            pidx[2 * e] = pairs[2 * e];
            pidx[2 * e + 1] = pairs[2 * e + 1];
        }
    __syncthreads();
    double* acc = p_smem ? pacc : gacc;
    const int32_t* pr = p_smem ? pidx : pairs;
    // the normals of the next iteration are loaded while this one computes
    double xn[NS + 1];
    if (i < N) {
        const double* nz = noise + (int64_t)r * (NS + 1) * Np + i;
#pragma unroll
        for (int a = 0; a < NS + 1; ++a) xn[a] = nz[(int64_t)a * Np];
    }
    for (int it = 0; it < iters; ++it) {
        const bool pro = prologue && it == 0;
        double xi[NS + 1];
#pragma unroll
        for (int a = 0; a < NS + 1; ++a) xi[a] = xn[a];
        if (i < N && it + 1 < iters) {
            const double* nz = noise + ((int64_t)(it + 1) * R + r) * (NS + 1) * Np + i;
#pragma unroll
            for (int a = 0; a < NS + 1; ++a) xn[a] = nz[(int64_t)a * Np];
        }
        double mq = 0.0;
        if (i < N) {
            // four independent partial sums: the FP64 latency chain is a quarter as long
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int k = 0;
            if (m_smem) {
                for (; k + 4 <= N; k += 4) {
                    a0 = fma(mt[(int64_t)k * Np + i], qs[k], a0);
                    a1 = fma(mt[(int64_t)(k + 1) * Np + i], qs[k + 1], a1);
                    a2 = fma(mt[(int64_t)(k + 2) * Np + i], qs[k + 2], a2);
                    a3 = fma(mt[(int64_t)(k + 3) * Np + i], qs[k + 3], a3);
                }
                for (; k < N; ++k) a0 = fma(mt[(int64_t)k * Np + i], qs[k], a0);
            } else {
                const double* mi = M + (int64_t)i * Np;
                for (; k + 4 <= N; k += 4) {
                    a0 = fma(mi[k], qs[k], a0);
                    a1 = fma(mi[k + 1], qs[k + 1], a1);
                    a2 = fma(mi[k + 2], qs[k + 2], a2);
                    a3 = fma(mi[k + 3], qs[k + 3], a3);
                }
                for (; k < N; ++k) a0 = fma(mi[k], qs[k], a0);
            }
            mq = (a0 + a1) + (a2 + a3);
        }
        __syncthreads();   // all reads of qs done before it is overwritten
        if (i < N) {
            if (!pro) {
                // end of the step, sample, start of the next: the two O half-steps jointly
                v[0] = fma(-g.hdt, mq, v[0]);
                const double pmid = o_sample64<NS>(v, g, xi);
                o_apply64<NS>(v, g.D2, xi);
                xs[i] = observable ? qi : pmid;
            } else {
                o_apply64<NS>(v, g.T, xi);
            }
            v[0] = fma(-g.hdt, mq, v[0]);
            qi = fma(g.dt, v[0], qi);
            qs[i] = qi;
        }
        __syncthreads();
        const int f = prologue ? it - 1 : it;   // index of this fused launch in the segment
        if (!pro && f >= acc_from) {
#pragma unroll 4
            for (int e = i; e < npairs; e += blockDim.x)
                acc[e] = fma(xs[pr[2 * e]], xs[pr[2 * e + 1]], acc[e]);
        }
        // xs is rewritten only after the next iteration's barrier
    }
    if (p_smem) {
        __syncthreads();
        for (int e = i; e < npairs; e += blockDim.x) gacc[e] = pacc[e];
    }
    if (i < N) {
        q[base + i] = qi;
        p[base + i] = v[0];
#pragma unroll
        for (int a = 1; a < NS; ++a) s[(a - 1) * plane + base + i] = v[a];
    }
}

// Small problems (N <= 32): the FP64 units of an SM sit in its four sub-partitions and a
// warp issues to one of them, so one warp per replica uses a quarter of the SM's FP64
// rate.  Here WARPS warps share each replica's work: warp w forms the force over columns
// k = Cw .. Cw + C - 1 (C = 32 / WARPS) and the O-step outputs o = w, w + WARPS, ... (pmid
// and out[0..NS) are NS + 1 rows of the joint update, their noise terms premixed by
// fp64_noise_kernel); lane = dof.  State in shared memory, double-buffered between steps;
// two barriers per step.
template <int NS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
fp64_small_kernel(GleF64 g, int N, int Np, const double* __restrict__ M, double* __restrict__ q,
                  double* __restrict__ p, double* __restrict__ s, const double* __restrict__ noise,
                  int iters, int prologue, int observable, const int32_t* __restrict__ pairs,
                  int npairs, double* __restrict__ partial, int acc_from) {
    extern __shared__ double sh[];
    double* qs = sh;                              // [32]
    double* xs = qs + 32;                         // [32]
    double* fpart = xs + 32;                      // [WARPS][32]
    double* vs = fpart + WARPS * 32;              // [2][NS][32]
    double* mt = vs + 2 * NS * 32;                // [32][32] (M transposed)
    double* pacc = mt + 32 * 32;                  // [npairs]
    int32_t* pidx = reinterpret_cast<int32_t*>(pacc + npairs);
    const int r = blockIdx.x, R = gridDim.x;
    const int warp = threadIdx.x >> 5, i = threadIdx.x & 31, tid = threadIdx.x;
    const int64_t base = (int64_t)r * Np;
    const int64_t plane = (int64_t)R * Np;
    double* gacc = partial + (int64_t)r * npairs;
    if (warp == 0) {
        qs[i] = i < N ? q[base + i] : 0.0;
        vs[i] = i < N ? p[base + i] : 0.0;
#pragma unroll
        for (int a = 1; a < NS; ++a) vs[a * 32 + i] = i < N ? s[(a - 1) * plane + base + i] : 0.0;
    }
    constexpr int kThreads = WARPS * 32;
    for (int e = tid; e < 32 * 32; e += kThreads) {
        const int row = e / 32, k = e % 32;
        mt[k * 32 + row] = (row < N && k < N) ? M[(int64_t)row * Np + k] : 0.0;
    }
    for (int e = tid; e < npairs; e += kThreads) {
        pacc[e] = gacc[e];
        pidx[2 * e] = pairs[2 * e];
        pidx[2 * e + 1] = pairs[2 * e + 1];
    }
    double zn[NS + 1];
    {
        const double* nz = noise + (int64_t)r * (NS + 1) * Np + (i < N ? i : 0);
#pragma unroll
        for (int a = 0; a < NS + 1; ++a) zn[a] = nz[(int64_t)a * Np];
    }
    __syncthreads();
    int cb = 0;
    for (int it = 0; it < iters; ++it) {
        const bool pro = prologue && it == 0;
        double z[NS + 1];
#pragma unroll
        for (int a = 0; a < NS + 1; ++a) z[a] = zn[a];
        if (it + 1 < iters) {
            const double* nz = noise + ((int64_t)(it + 1) * R + r) * (NS + 1) * Np + (i < N ? i : 0);
#pragma unroll
            for (int a = 0; a < NS + 1; ++a) zn[a] = nz[(int64_t)a * Np];
        }
        // force, 32 / WARPS columns per warp in two FMA chains
        {
            constexpr int C = 32 / WARPS;
            double f0 = 0.0, f1 = 0.0;
#pragma unroll
            for (int k = 0; k < C; k += 2) {
                f0 = fma(mt[(warp * C + k) * 32 + i], qs[warp * C + k], f0);
                f1 = fma(mt[(warp * C + k + 1) * 32 + i], qs[warp * C + k + 1], f1);
            }
            fpart[warp * 32 + i] = f0 + f1;
        }
        __syncthreads();
        double mq;
        if (WARPS == 4) {
            mq = (fpart[i] + fpart[32 + i]) + (fpart[64 + i] + fpart[96 + i]);
        } else {
            mq = ((fpart[i] + fpart[32 + i]) + (fpart[64 + i] + fpart[96 + i])) +
                 ((fpart[128 + i] + fpart[160 + i]) + (fpart[192 + i] + fpart[224 + i]));
        }
        const double* vc = vs + cb * NS * 32;
        double* vn = vs + (cb ^ 1) * NS * 32;
        double v[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) v[a] = vc[a * 32 + i];
        if (!pro) v[0] = fma(-g.hdt, mq, v[0]);   // B(dt/2), end of the step (not in the prologue)
#pragma unroll
        for (int o = 0; o <= NS; ++o) {
            if (o % WARPS != warp) continue;
            if (o == 0) {
                if (!pro) {
                    double u = z[0];                       // premixed noise of the sample
#pragma unroll
                    for (int b = 0; b < NS; ++b) u = fma(g.T[b], v[b], u);
                    if (!observable) xs[i] = v[0] + u;
                }
                continue;
            }
            const int a = o - 1;
            double acc = z[a + 1];                         // premixed noise term
            const double* D = pro ? g.T : g.D2;
#pragma unroll
            for (int b = 0; b < NS; ++b) acc = fma(D[a * kMaxNs + b], v[b], acc);
            double va = v[a] + acc;
            if (a == 0) {
                // B(dt/2) and A(dt) of the next step; the sample of q is the position before A
                va = fma(-g.hdt, mq, va);
                const double qold = qs[i];
                if (!pro && observable) xs[i] = qold;
                qs[i] = fma(g.dt, va, qold);
            }
            vn[a * 32 + i] = va;
        }
        __syncthreads();
        const int f = prologue ? it - 1 : it;
        if (!pro && f >= acc_from)
            for (int e = tid; e < npairs; e += kThreads)
                pacc[e] = fma(xs[pidx[2 * e]], xs[pidx[2 * e + 1]], pacc[e]);
        cb ^= 1;
    }
    __syncthreads();
    for (int e = tid; e < npairs; e += kThreads) gacc[e] = pacc[e];
    if (warp == 0 && i < N) {
        q[base + i] = qs[i];
        p[base + i] = vs[cb * NS * 32 + i];
#pragma unroll
        for (int a = 1; a < NS; ++a) s[(a - 1) * plane + base + i] = vs[cb * NS * 32 + a * 32 + i];
    }
}

cudaError_t launch_fp64_noise(int ns, const GleF64& g, int64_t N, int64_t Np, int64_t R,
                              uint32_t kappa0, int64_t iters, int prologue, double* xi,
                              cudaStream_t st) {
    if (iters <= 0) return cudaSuccess;
    const int64_t total = iters * (R / 2 + 1) * N;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
#define FTH_F64N_CASE(NSV)                                                                  \
    case NSV:                                                                               \
        fp64_noise_kernel<NSV><<<grid, 256, 0, st>>>(g, (int)N, (int)Np, (int)R, kappa0,    \
                                                     (int)iters, prologue, xi);             \
        break;
    switch (ns) {
        FTH_F64N_CASE(1)
        FTH_F64N_CASE(2)
        FTH_F64N_CASE(3)
        FTH_F64N_CASE(4)
        FTH_F64N_CASE(5)
        default: return cudaErrorInvalidValue;
    }
#undef FTH_F64N_CASE
    return cudaGetLastError();
}

// Warps per replica of the N <= 32 kernel: eight split the force columns four ways finer
// and give each of the NS + 1 O outputs its own warp.
constexpr int kFp64Warps = 8;

cudaError_t launch_fp64_dense(int ns, const GleF64& g, int64_t N, int64_t Np, int64_t R,
                              const double* M, double* q, double* p, double* s,
                              const double* noise, int64_t nsteps, int primed_in, int observable,
                              const int32_t* pairs, int64_t npairs, double* partial,
                              int64_t acc_from, cudaStream_t st) {
    const int prologue = primed_in ? 0 : 1;
    const int iters = (int)nsteps + prologue;
    if (iters <= 0) return cudaSuccess;
    constexpr size_t kBudget = 200 * 1024;
    const size_t small_bytes = sizeof(double) * (32 * (2 + kFp64Warps) + 2 * (size_t)ns * 32 +
                                                 32 * 32) +
                               (size_t)npairs * 16;
    if (N <= 32 && small_bytes <= kBudget) {
#define FTH_F64S_CASE(NSV)                                                                  \
    case NSV:                                                                               \
        cudaFuncSetAttribute(fp64_small_kernel<NSV, kFp64Warps>,                            \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBudget);    \
        fp64_small_kernel<NSV, kFp64Warps><<<(unsigned)R, kFp64Warps * 32, small_bytes, st>>>( \
            g, (int)N, (int)Np, M, q, p, s, noise, iters, prologue, observable, pairs,      \
            (int)npairs, partial, (int)acc_from);                                           \
        break;
        switch (ns) {
            FTH_F64S_CASE(1)
            FTH_F64S_CASE(2)
            FTH_F64S_CASE(3)
            FTH_F64S_CASE(4)
            FTH_F64S_CASE(5)
            default: return cudaErrorInvalidValue;
        }
#undef FTH_F64S_CASE
        return cudaGetLastError();
    }
    const int threads = (int)std::max<int64_t>(32, ((N + 31) / 32) * 32);
    // shared memory: q and x always; then the pairs (16 B each) and M when they fit
    size_t shmem = sizeof(double) * 2 * (size_t)Np;
    const size_t pbytes = (size_t)npairs * 16, mbytes = (size_t)N * Np * 8;
    const int p_smem = shmem + pbytes <= kBudget ? 1 : 0;
    if (p_smem) shmem += pbytes;
    const int m_smem = shmem + mbytes <= kBudget ? 1 : 0;
    if (m_smem) shmem += mbytes;
    // noise holds the normals of the segment's kick indices (the prologue's first)
#define FTH_F64_CASE(NSV)                                                                   \
    case NSV:                                                                               \
        cudaFuncSetAttribute(fp64_dense_kernel<NSV>,                                        \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBudget);    \
        fp64_dense_kernel<NSV><<<(unsigned)R, threads, shmem, st>>>(                        \
            g, (int)N, (int)Np, M, q, p, s, noise, iters, prologue, observable, pairs,      \
            (int)npairs, partial, (int)acc_from, m_smem, p_smem);                           \
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
