// Problem-pool descriptors shared by the pool's host runtime and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fth_internal.h"

namespace fth {

// One problem slot, resident in device memory; the kernels read everything they need
// from here (constants, buffers, counters), the accumulate kernel advances the counters.
struct PoolDesc {
    GleF32 g;               // D = T - I, S, dt, Philox keys (round keys), replica offset
    int kind;               // 0 dense, 1 CSR
    int n, np;              // order; dense: order padded to 128
    int ns;                 // s + 1
    int observable;
    int npairs;
    int live;
    int sym;                // dense BF16: M stored as its upper 128 x 128 blocks only
    int64_t burnin, block;
    // dense force operands.  TF32: M blocked and pre-swizzled in 128-byte K slices
    // ([np/128][np/32][128][128 B]).  BF16 (sym): the upper blocks (I <= J) in packed
    // order, each as four 64 x 64 sub-tiles (row half a, column half b) at
    // (2 b + a) * 8 KiB, 128-byte rows, 16-byte chunk c of row r at c ^ (r & 7); a lower
    // block is read as the transpose of its mirror (MN-major A operand).
    // q^T slices ([np/KS][R][128 B]).
    uint8_t* a_hi;
    uint8_t* a_lo;
    uint8_t* bt_hi;
    uint8_t* bt_lo;
    float* mq;              // M q, [n][R]
    float* q[2];            // positions [n][R] (CSR: ping-pong, q[cur] current)
    float* p;
    float* s;               // ns - 1 planes of [n][R]
    const int32_t* rowptr;  // CSR
    const int32_t* col;
    const float* val;
    float* x;               // this step's sample [n][R]
    const int32_t* pairs;   // 2 * npairs, local indices
    float* partial;         // block partial sums
    double* mean;           // Welford mean of the block means
    double* m2;
    // counters, advanced on the device by the accumulate kernel
    int64_t t, nsamp, inblock, nblocks;
    int primed, cur;
    int done;               // accumulate items of this step finished (reset by the last)
    int pad1;
};

struct PoolForceItem {
    int problem;
    int rb;                 // 128-row block
};

struct PoolRowItem {
    int problem;
    int row0;               // first of 32 rows
};

// Accumulate work: pairs [e0, e1) of one problem; the problem has `nchunks` items.
struct PoolAccItem {
    int problem;
    int e0, e1;
    int nchunks;
};
constexpr int kPoolAccChunk = 256;   // pairs per item (one thread each)

cudaError_t launch_pool_force(int kind, int rn, int variant, const PoolDesc* desc,
                              const PoolForceItem* items, int nitems, int grid, uint32_t* err,
                              cudaStream_t st);
int pool_force_max_ctas_per_sm(int kind, int rn, int variant);
cudaError_t launch_pool_convert(const void* src, int f64, int n, int np, int r0, int nr, int kind,
                                uint8_t* a_hi, uint8_t* a_lo, cudaStream_t st);
cudaError_t launch_pool_progress(const PoolDesc* desc, const int* live, int nlive, double* out,
                                 cudaStream_t st);
constexpr size_t kPoolStageBytes = size_t(16) << 20;   // host-to-device staging of M rows
constexpr int kPoolGleVariants = 4;
cudaError_t launch_pool_gle(int variant, const PoolDesc* desc, const PoolRowItem* items,
                            int nitems, int RN, int kind, int ns, const GleF32& gk,
                            cudaStream_t st);
cudaError_t launch_pool_csr(const PoolDesc* desc, const PoolRowItem* items, int nitems, int RN,
                            int ns, const GleF32& gk, cudaStream_t st);
cudaError_t launch_pool_accum(PoolDesc* desc, const PoolAccItem* items, int nitems, int RN,
                              uint32_t* err, cudaStream_t st);

}  // namespace fth
