// Device helpers of the GLE step: counter-based noise and the O / B / A updates.
//
// Noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor S-box on a 4x32-bit counter with a 2x32-bit key bumped by the Weyl
// constants between rounds.  Replicas are paired: for kick index kappa, dof i and pair
// j, call k uses counter (kappa, i, j, k) and key (seed_lo, seed_hi), and the calls
// form one stream of normals, four per call.  Box-Muller turns each uint32 pair (a, b)
// into two normals rho*cos(2 pi u_b), rho*sin(2 pi u_b) with rho = sqrt(-2 ln u_a) and
// u(x) = ((x >> 9) * 2 + 1) * 2^-24, exact in FP32 and never 0 or 1.  Global replica g
// (index plus the replica offset) belongs to pair g / 2 and takes stream positions
// (g mod 2) W .. (g mod 2) W + W - 1, W = ns + 1.  A fused launch (end of step kappa-1
// and start of step kappa) uses those W normals of kappa for its two O half-steps,
// drawn jointly (gle_fused); a launch with one half-step (the prologue) uses the first
// ns of them.
#pragma once

#include <stdint.h>

#include "fth_internal.h"

namespace fth {

// Philox4x32-10 with the round keys precomputed (rk[2j], rk[2j+1] = key + j * Weyl),
// e.g. from a kernel parameter, so the XORs take them as constant operands.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* rk) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * round], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * round + 1], (uint32_t)p0);
    }
    return c;
}

// One 32x32 -> 64-bit multiply per S-box gives both halves.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// u = ((x >> 9) * 2 + 1) * 2^-24, built from bits: 1 + (x >> 9) 2^-23 is exact as a
// float, and subtracting 1 - 2^-24 is exact (Sterbenz: both operands within a factor 2).
__device__ __forceinline__ float open_unit(uint32_t x) {
    return __uint_as_float(0x3F800000u | (x >> 9)) - 0.999999940395355224609375f;
}

// rho = sqrt(-2 ln u_a) with the accurate logf (near u = 1 the approximate log's
// absolute error would dominate rho); the angle 2 pi u_b is shifted by pi into
// (-pi, pi), where the hardware sine/cosine are accurate to ~2^-21 absolute, and the
// shift is undone by the sign: cos(2 pi u) = -cos(2 pi (u - 1/2)), same for sin.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
    const float r2 = -2.0f * logf(open_unit(a));
    const float rho = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    float sn, cs;
    __sincosf(6.28318530717958648f * (open_unit(b) - 0.5f), &sn, &cs);
    z0 = -rho * cs;
    z1 = -rho * sn;
}

// The W = NS + 1 normals of both replicas of pair j (global replicas 2j and 2j + 1):
// all four words of each of the ceil(2W / 4) calls.
template <int NS>
__device__ __forceinline__ void gle_normals_pair(uint32_t kappa, uint32_t i, uint32_t j,
                                                 const uint32_t* rk, float (&xa)[NS + 1],
                                                 float (&xb)[NS + 1]) {
    constexpr int W = NS + 1;
    constexpr int kCalls = (2 * W + 3) / 4;
#pragma unroll
    for (int k = 0; k < kCalls; ++k) {
        const uint4 x = philox4x32_10_rk(make_uint4(kappa, i, j, (uint32_t)k), rk);
        float z[4];
        box_muller(x.x, x.y, z[0], z[1]);
        if (4 * k + 2 < 2 * W) box_muller(x.z, x.w, z[2], z[3]);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int pos = 4 * k + t;
            if (pos < W) xa[pos] = z[t];
            else if (pos < 2 * W) xb[pos - W] = z[t];
        }
    }
}

// Half H (0: even replica, 1: odd) of pair j alone: only the calls and Box-Muller
// transforms that cover stream positions H W .. H W + W - 1.
template <int NS, int H>
__device__ __forceinline__ void gle_normals_half(uint32_t kappa, uint32_t i, uint32_t j,
                                                 const uint32_t* rk, float (&xi)[NS + 1]) {
    constexpr int W = NS + 1;
    constexpr int p0 = H * W, p1 = H * W + W;     // [p0, p1)
#pragma unroll
    for (int k = p0 / 4; k <= (p1 - 1) / 4; ++k) {
        const uint4 x = philox4x32_10_rk(make_uint4(kappa, i, j, (uint32_t)k), rk);
        float z[4];
        if (4 * k + 2 > p0 && 4 * k < p1) box_muller(x.x, x.y, z[0], z[1]);
        if (4 * k + 4 > p0 && 4 * k + 2 < p1) box_muller(x.z, x.w, z[2], z[3]);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int pos = 4 * k + t;
            if (pos >= p0 && pos < p1) xi[pos - p0] = z[t];
        }
    }
}

// The NS + 1 normals of one global replica g alone.
template <int NS>
__device__ __forceinline__ void gle_normals(uint32_t kappa, uint32_t i, uint32_t g,
                                            const uint32_t* rk, float (&xi)[NS + 1]) {
    if (g & 1u) gle_normals_half<NS, 1>(kappa, i, g >> 1, rk, xi);
    else gle_normals_half<NS, 0>(kappa, i, g >> 1, rk, xi);
}

// The normals of two consecutive global replicas g and g + 1: one pair stream when they
// form a pair (g even), else each alone.
template <int NS>
__device__ __forceinline__ void gle_normals_two(uint32_t kappa, uint32_t i, uint32_t g,
                                                const uint32_t* rk, float (&xa)[NS + 1],
                                                float (&xb)[NS + 1]) {
    if ((g & 1u) == 0u) {
        gle_normals_pair<NS>(kappa, i, g >> 1, rk, xa, xb);
    } else {
        gle_normals_half<NS, 1>(kappa, i, g >> 1, rk, xa);
        gle_normals_half<NS, 0>(kappa, i, (g >> 1) + 1u, rk, xb);
    }
}

// v <- T v + S xi on v = (p, s_1..s_{NS-1}), with T passed as D = T - I: the
// increment D v + S xi is formed first and added to v once, so rounding D (whose
// entries are O(dt |A_p|)) costs far less than rounding T itself would.
template <int NS, typename Real>
__device__ __forceinline__ void o_half(Real (&v)[NS], const Real* D, const Real* S,
                                       const Real* xi) {
    Real out[NS];
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        Real acc = Real(0);
#pragma unroll
        for (int b = 0; b < NS; ++b) acc = fma(D[a * kMaxNs + b], v[b], acc);
#pragma unroll
        for (int b = 0; b <= a; ++b) acc = fma(S[a * kMaxNs + b], xi[b], acc);
        out[a] = v[a] + acc;
    }
#pragma unroll
    for (int a = 0; a < NS; ++a) v[a] = out[a];
}

// The two O half-steps around the end-of-step sample, drawn jointly: with v the state
// after the end-of-step kick, the sample (observable p) is (T v)_0 + (L zeta)_0 and the
// next state T T v + (L zeta)_1..NS, zeta = NS + 1 normals.  Increment form as o_half.
template <int NS, typename Real, typename G>
__device__ __forceinline__ void o_joint(Real (&v)[NS], const G& g, const Real* zeta,
                                        Real& pmid) {
    Real inc = g.L[0] * zeta[0];
#pragma unroll
    for (int b = 0; b < NS; ++b) inc = fma(g.T[b], v[b], inc);
    pmid = v[0] + inc;
    Real out[NS];
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        Real acc = Real(0);
#pragma unroll
        for (int b = 0; b < NS; ++b) acc = fma(g.D2[a * kMaxNs + b], v[b], acc);
#pragma unroll
        for (int b = 0; b <= a + 1; ++b) acc = fma(g.L[(a + 1) * kMaxNs1 + b], zeta[b], acc);
        out[a] = v[a] + acc;
    }
#pragma unroll
    for (int a = 0; a < NS; ++a) v[a] = out[a];
}

// One fused launch on one (i, r): mq = (M q)_i at the current positions.
//   end + start : p += -hdt mq;  both O half-steps jointly, sample between;
//                 p += -hdt mq;  q += dt p
//   start only  : O(zeta[0..NS));  p += -hdt mq;  q += dt p       (prologue)
//   end only    : p += -hdt mq;  O(zeta[0..NS));  sample
template <int NS>
__device__ __forceinline__ void gle_fused(float& q, float (&v)[NS], float mq, const GleF32& g,
                                          const float (&xi)[NS + 1], int flags, int observable,
                                          float& sample) {
    if ((flags & kDoEnd) && (flags & kDoStart)) {
        v[0] = fmaf(-g.hdt, mq, v[0]);
        float pmid;
        o_joint<NS, float>(v, g, xi, pmid);
        sample = observable ? q : pmid;
        v[0] = fmaf(-g.hdt, mq, v[0]);
        q = fmaf(g.dt, v[0], q);
        return;
    }
    if (flags & kDoEnd) {
        v[0] = fmaf(-g.hdt, mq, v[0]);
        o_half<NS, float>(v, g.T, g.S, xi);
        sample = observable ? q : v[0];
    }
    if (flags & kDoStart) {
        o_half<NS, float>(v, g.T, g.S, xi);
        v[0] = fmaf(-g.hdt, mq, v[0]);
        q = fmaf(g.dt, v[0], q);
    }
}

// The steady-state update (end and start) of two replicas at once, one in each lane of
// float2 registers: the same sequence of roundings as gle_fused, issued as packed FP32
// instructions (each lane of fma.rn.f32x2 rounds as fmaf does), so both lanes equal
// gle_fused's results bit for bit in half the floating-point instructions.
template <int NS>
__device__ __forceinline__ void o_joint2(float2 (&v)[NS], const GleF32& g,
                                         const float2 (&zeta)[NS + 1], float2& pmid) {
    float2 inc = __fmul2_rn(g.Lx2[0], zeta[0]);
#pragma unroll
    for (int b = 0; b < NS; ++b) inc = __ffma2_rn(g.T0x2[b], v[b], inc);
    pmid = __fadd2_rn(v[0], inc);
    float2 out[NS];
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < NS; ++b) acc = __ffma2_rn(g.D2x2[a * kMaxNs + b], v[b], acc);
#pragma unroll
        for (int b = 0; b <= a + 1; ++b) acc = __ffma2_rn(g.Lx2[(a + 1) * kMaxNs1 + b], zeta[b], acc);
        out[a] = __fadd2_rn(v[a], acc);
    }
#pragma unroll
    for (int a = 0; a < NS; ++a) v[a] = out[a];
}

template <int NS>
__device__ __forceinline__ void gle_fused2(float2& q, float2 (&v)[NS], float2 mq, const GleF32& g,
                                           const float2 (&zeta)[NS + 1], int observable,
                                           float2& sample) {
    v[0] = __ffma2_rn(g.mhdt2, mq, v[0]);
    float2 pmid;
    o_joint2<NS>(v, g, zeta, pmid);
    sample = observable ? q : pmid;
    v[0] = __ffma2_rn(g.mhdt2, mq, v[0]);
    q = __ffma2_rn(g.dt2, v[0], q);
}

// One thread's four consecutive replicas r0 .. r0 + 3 of dof i, held as float4 (q, the
// NS momentum planes, mq): two Philox pair streams; in the steady state a pair whose
// replicas are both below R takes the packed update, any other replica gle_fused.
template <int NS>
__device__ __forceinline__ void gle_quad(float4& q4, float4 (&v4)[NS], const float4& mq4,
                                         const GleF32& g, uint32_t kappa, uint32_t i, int r0,
                                         int R, int flags, int observable, float (&samp)[4]) {
    float* qa = reinterpret_cast<float*>(&q4);
    const float* mqa = reinterpret_cast<const float*>(&mq4);
#pragma unroll
    for (int e = 0; e < 4; e += 2) {
        if (r0 + e >= R) continue;
        float xa[NS + 1], xb[NS + 1];
        gle_normals_two<NS>(kappa, i, (uint32_t)(r0 + e) + g.roff, g.rk, xa, xb);
        if ((flags & kDoEnd) && (flags & kDoStart) && r0 + e + 1 < R) {
            float2 zeta[NS + 1];
#pragma unroll
            for (int k = 0; k <= NS; ++k) zeta[k] = make_float2(xa[k], xb[k]);
            float2 v[NS];
#pragma unroll
            for (int a = 0; a < NS; ++a) v[a] = reinterpret_cast<float2*>(&v4[a])[e >> 1];
            float2 q = reinterpret_cast<float2*>(&q4)[e >> 1];
            float2 sm;
            gle_fused2<NS>(q, v, reinterpret_cast<const float2*>(&mq4)[e >> 1], g, zeta,
                           observable, sm);
#pragma unroll
            for (int a = 0; a < NS; ++a) reinterpret_cast<float2*>(&v4[a])[e >> 1] = v[a];
            reinterpret_cast<float2*>(&q4)[e >> 1] = q;
            samp[e] = sm.x;
            samp[e + 1] = sm.y;
            continue;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ee = e + h;
            if (r0 + ee >= R) continue;
            float v[NS];
#pragma unroll
            for (int a = 0; a < NS; ++a) v[a] = reinterpret_cast<float*>(&v4[a])[ee];
            if (h == 0) gle_fused<NS>(qa[ee], v, mqa[ee], g, xa, flags, observable, samp[ee]);
            else gle_fused<NS>(qa[ee], v, mqa[ee], g, xb, flags, observable, samp[ee]);
#pragma unroll
            for (int a = 0; a < NS; ++a) reinterpret_cast<float*>(&v4[a])[ee] = v[a];
        }
    }
}

}  // namespace fth
