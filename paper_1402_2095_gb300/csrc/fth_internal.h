// Internal declarations shared by the host runtime and the kernels of libfth.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fth.h"

namespace fth {

constexpr int kMaxNs = 5;          // s + 1 <= 5 (s <= 4 auxiliary momenta)
constexpr int kTile = 128;         // tcgen05 M tile (rows per CTA) and SYRK tile edge

// O half-step constants in FP32 (the FP64 originals are built on the host).
// T holds D = T - I (the increment form used by the O half-step), S is lower triangular.
// O half-step constants.  T holds D = T - I (the increment form keeps FP32 rounding
// small), S the noise factor of one half-step.  A fused launch applies the two
// half-steps around the end-of-step sample jointly: D2 = T T - I, and L
// ([ns+1][ns+1], lower, row stride kMaxNs + 1) factors the joint covariance of the
// sample's noise and the two half-steps' noise (ns + 1 normals).
constexpr int kMaxNs1 = kMaxNs + 1;
struct GleF32 {
    float T[kMaxNs * kMaxNs];
    float S[kMaxNs * kMaxNs];
    float D2[kMaxNs * kMaxNs];
    float L[kMaxNs1 * kMaxNs1];
    float dt, hdt;
    uint32_t key0, key1;
    uint32_t roff;   // replica offset in the noise counter
    uint32_t rk[20]; // Philox round keys: key + j * (0x9E3779B9, 0xBB67AE85), j = 0..9
    // The constants of the two-replica update (gle_fused2), each duplicated into both
    // lanes: a packed FP32 instruction reads such a pair as one 64-bit operand.
    float2 D2x2[kMaxNs * kMaxNs];
    float2 Lx2[kMaxNs1 * kMaxNs1];
    float2 T0x2[kMaxNs];   // row 0 of D = T - I
    float2 mhdt2, dt2;     // -dt/2 and dt
};

// Fills g.rk from g.key0, g.key1, and the duplicated pairs from D2, L, T, hdt and dt
// (call once those are set).
inline void set_round_keys(GleF32& g) {
    for (int j = 0; j < 10; ++j) {
        g.rk[2 * j] = g.key0 + (uint32_t)j * 0x9E3779B9u;
        g.rk[2 * j + 1] = g.key1 + (uint32_t)j * 0xBB67AE85u;
    }
    for (int k = 0; k < kMaxNs * kMaxNs; ++k) g.D2x2[k] = make_float2(g.D2[k], g.D2[k]);
    for (int k = 0; k < kMaxNs1 * kMaxNs1; ++k) g.Lx2[k] = make_float2(g.L[k], g.L[k]);
    for (int k = 0; k < kMaxNs; ++k) g.T0x2[k] = make_float2(g.T[k], g.T[k]);
    g.mhdt2 = make_float2(-g.hdt, -g.hdt);
    g.dt2 = make_float2(g.dt, g.dt);
}

struct GleF64 {
    double T[kMaxNs * kMaxNs];
    double S[kMaxNs * kMaxNs];
    double D2[kMaxNs * kMaxNs];
    double L[kMaxNs1 * kMaxNs1];
    double dt, hdt;
    uint32_t key0, key1;
    uint32_t roff;
};

// Fills the O half-step constants of both precisions (either may be NULL) from the
// FP64 propagator T, S ([ns][ns], row-major): D = T - I, S, D2 = T T - I and the
// joint factor L of the two half-steps around the end-of-step sample.
void fill_gle_constants(int ns, const double* T, const double* S, GleF32* g32, GleF64* g64);

// Bits of the device error word.
enum : uint32_t { kErrTimeout = 1u, kErrNonFinite = 2u };

// Dense M preparation on the device (k_prepare.cu): target layouts and validation flags.
enum : int { kPrepF64 = 0, kPrepF32 = 1, kPrepTf32 = 2, kPrepBf16x3 = 3 };
enum : uint32_t { kPrepNotSpd = 1u, kPrepNonFinite = 2u };
// Rows r0 .. r0 + nr - 1 of a row-major n x n matrix at src (device memory holding just
// those rows; FP64 if f64, else FP32) into the layout's buffer(s) hi (and lo for BF16x3)
// of order Np; atomically ORs kPrepNotSpd / kPrepNonFinite into *flags.
cudaError_t launch_dense_prepare(const void* src, int f64, int64_t n, int64_t r0, int64_t nr,
                                 int64_t Np, int layout, void* hi, void* lo, uint32_t* flags,
                                 cudaStream_t st);

// Flags of the dense element-wise GLE kernel.  kSampleBf16: stage the samples in a BF16
// stack, rounded to nearest, for the tensor-core accumulation pass (kind::f16 operands:
// twice the TF32 MMA rate and half the bytes; the rounding errors average out over the
// samples up to a bias of order 1e-5 of each element).
// kZeroMQ: write zeros over MQ after reading it (the force adds its partial sums into MQ).
enum : int { kDoEnd = 1, kDoStart = 2, kDoSample = 4, kSampleBf16 = 8, kZeroMQ = 16 };

// Operand copies of q the element-wise kernel writes for the force GEMM.
enum : int { kOpNone = 0, kOpTf32 = 1, kOpBf16x2 = 2 };

// ------------------------------------------------------------------ kernels
// Dense path, state planes [Np][Rp] FP32 (replica fastest), MQ = M q (positive).
cudaError_t launch_dense_gle(int ns, const GleF32& g, int64_t N, int64_t R, int64_t Rp,
                             float* MQ, int mq_planes, float* q, float* p, float* s,
                             uint32_t kappa,
                             int flags, int observable, float* ps, int64_t ps_ld, int64_t slot,
                             int op_kind, void* op_hi, void* op_lo, int64_t Np,
                             cudaStream_t st);

// Planes of MQ the FP32 force writes (its K shares; the element-wise step sums them).
int sgemm_force_planes(int64_t Rp);
cudaError_t launch_sgemm_force(const float* M, int64_t ldm, const float* q, int64_t Rp,
                               float* MQ, int64_t N, cudaStream_t st);

// CSR path: fused SpMM + GLE (force on q_in, positions written to q_out).
cudaError_t launch_csr_step(int ns, const GleF32& g, int64_t N, int64_t R, int64_t Rp,
                            const int32_t* rowptr, const int32_t* col, const float* val,
                            const float* q_in, float* q_out, float* p, float* s,
                            uint32_t kappa, int flags, int observable, float* ps,
                            int64_t ps_ld, int64_t slot, cudaStream_t st);

// Accumulation: partial[e] += sum_{c < ncols} ps[i_e][c] * ps[j_e][c].
cudaError_t launch_pair_accum(const float* ps, int64_t ps_ld, int64_t ncols,
                              const int32_t* pairs, int64_t npairs, float* partial,
                              cudaStream_t st);

// SYRK over the staged samples into tile-packed FP32 partials (upper tiles I <= J).
cudaError_t launch_syrk_fp32(const float* ps, int64_t ps_ld, int64_t ncols, int64_t Np,
                             float* tiles, cudaStream_t st);

// FP64 Welford update with one block mean per element: b = partial * inv_count.
cudaError_t launch_flush(float* partial, double* mean, double* m2, int64_t count,
                         double inv_count, double nb, uint32_t* err, cudaStream_t st);
cudaError_t launch_flush64(double* partial, int64_t R, int64_t stride, double* mean, double* m2,
                           int64_t count, double inv_count, double nb, uint32_t* err,
                           cudaStream_t st);

// Gather (mean, m2, partial) of requested elements into out[3 * k].
cudaError_t launch_gather(const int64_t* idx, int64_t k, const double* mean, const double* m2,
                          const float* partial32, const double* partial64, int64_t p64_R,
                          int64_t p64_stride, double* out, cudaStream_t st);

// Element (i, j) of the tile-packed layout -> flat index (host helper mirrored on device).
__host__ __device__ inline int64_t packed_index(int64_t i, int64_t j, int64_t nb_tiles) {
    if (i > j) { int64_t t = i; i = j; j = t; }
    const int64_t I = i / kTile, J = j / kTile;
    const int64_t tile = I * nb_tiles - (I * (I - 1)) / 2 + (J - I);
    return tile * (int64_t)kTile * kTile + (i % kTile) * kTile + (j % kTile);
}

// Pair accumulation grouped by row (CSR of partners); ncols must be supported.
bool pair_accum_rows_supported(int64_t ncols);
cudaError_t launch_pair_accum_rows(const float* ps, int64_t ps_ld, int64_t ncols,
                                   const int32_t* prow, const int32_t* pcol, const int32_t* pe,
                                   int64_t N, float* partial, cudaStream_t st);

// Linear functional of tracked elements: fold one completed block (see the kernel).
cudaError_t launch_functional_block(const float* partial32, const double* partial64, int64_t R,
                                    int64_t stride, const int64_t* idx, const double* w,
                                    int64_t nterms, double inv_count, double nb, double* acc,
                                    uint32_t* err, cudaStream_t st);

// Conversions used at create / set_state.
cudaError_t launch_round_tf32(float* x, int64_t n, cudaStream_t st);
cudaError_t launch_split_bf16(const float* x, int64_t n, void* hi, void* lo, cudaStream_t st);

// FP64 small dense path: the noise terms of a segment are generated ahead over the whole
// GPU (`xi`: [iters][R][ns + 1][Np], the normals already multiplied by the O half-steps'
// noise factors; `prologue`: the first kick is the prologue's single half-step), then one
// CTA per replica runs `nsteps` fused launches (plus the prologue when not primed).
cudaError_t launch_fp64_noise(int ns, const GleF64& g, int64_t N, int64_t Np, int64_t R,
                              uint32_t kappa0, int64_t iters, int prologue, double* xi,
                              cudaStream_t st);
cudaError_t launch_fp64_dense(int ns, const GleF64& g, int64_t N, int64_t Np, int64_t R,
                              const double* M, double* q, double* p, double* s,
                              const double* noise, int64_t nsteps, int primed_in, int observable,
                              const int32_t* pairs, int64_t npairs, double* partial,
                              int64_t acc_from, cudaStream_t st);

// tcgen05 / TMA kernels (sm_103a).
struct TcForce;   // opaque, holds the tensor maps
// MQ (may be NULL): the [Np][Rp] output, for the row-pair kernel's reduce-add map.
cudaError_t tc_force_prepare(TcForce** out, int kind, const void* A_hi, const void* A_lo,
                             const void* B_hi, const void* B_lo, int64_t Np, int64_t Rp,
                             int64_t N, int64_t R, float* MQ);
cudaError_t tc_force_run(const TcForce* tf, float* MQ, int64_t ldf, uint32_t* err,
                         cudaStream_t st);
void tc_force_free(TcForce* tf);
// Test hook: stall_ns > 0 makes later launches issue no copies and end through their
// timeout path after stall_ns (see fth_test_stall); 0 restores normal launches.
void tc_force_set_stall(TcForce* tf, uint64_t stall_ns);
// True when the force adds into MQ (TMA reduce-adds), so the reader must zero MQ after use.
bool tc_force_accumulates(const TcForce* tf);

struct TcSyrk;
cudaError_t tc_syrk_prepare(TcSyrk** out, const void* ps, int64_t Np, int64_t ps_ld,
                            float* tiles);
cudaError_t tc_syrk_run(const TcSyrk* ts, int64_t ncols, float* tiles, uint32_t* err,
                        cudaStream_t st);
void tc_syrk_free(TcSyrk* ts);

}  // namespace fth
