// Device-side preparation of a dense M for a context: validation (positive diagonal,
// finite entries: a symmetric positive-definite M, the Hessian of Eq. 5, has both) and
// conversion into the force kernel's operand layout, from the caller's row-major N x N
// matrix (FP32 or FP64) or a chunk of its rows already copied to the device.  The
// roundings are the integer bit operations of the host-side forms (TF32 round to nearest,
// ties away; BF16 round to nearest even, hi + lo split), so the operands do not depend on
// where they were made.
#include <stdint.h>

#include <algorithm>

#include "fth_internal.h"

namespace fth {
namespace {

__device__ __forceinline__ float tf32_rna_dev(float f) {
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7F800000u) != 0x7F800000u) {
        u += 0x1000u;
        u &= ~0x1FFFu;
    }
    return __uint_as_float(u);
}

__device__ __forceinline__ uint16_t bf16_rne_dev(float f) {
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);   // inf / nan
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Offset of element (i, j) of an Np x Np matrix stored as [Np/128][Np/ks][128][ks].
__device__ __forceinline__ int64_t blocked_at(int64_t i, int64_t j, int64_t Np, int64_t ks) {
    return (((i / 128) * (Np / ks) + j / ks) * 128 + (i % 128)) * ks + (j % ks);
}

// Rows r0 .. r0 + nr - 1 of M (src holds exactly those rows, row-major, n columns).
// Only elements (i < n, j < n) are written: the padding stays as the zeroed workspace.
__global__ void __launch_bounds__(256)
dense_prepare_kernel(const void* __restrict__ src, int f64, int64_t n, int64_t r0, int64_t nr,
                     int64_t Np, int layout, void* __restrict__ hi, void* __restrict__ lo,
                     uint32_t* __restrict__ flags) {
    const int64_t total = nr * n;
    uint32_t bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r0 + k / n, j = k % n;
        const double x = f64 ? static_cast<const double*>(src)[k]
                             : (double)static_cast<const float*>(src)[k];
        if (!isfinite(x)) bad |= kPrepNonFinite;
        if (i == j && !(x > 0.0)) bad |= kPrepNotSpd;
        switch (layout) {
            case kPrepF64:
                static_cast<double*>(hi)[i * Np + j] = x;
                break;
            case kPrepF32:
                static_cast<float*>(hi)[i * Np + j] = (float)x;
                break;
            case kPrepTf32:
                static_cast<float*>(hi)[blocked_at(i, j, Np, 32)] = tf32_rna_dev((float)x);
                break;
            default: {
                const float xf = (float)x;
                const uint16_t hb = bf16_rne_dev(xf);
                const int64_t at = blocked_at(i, j, Np, 64);
                static_cast<uint16_t*>(hi)[at] = hb;
                static_cast<uint16_t*>(lo)[at] = bf16_rne_dev(xf - __uint_as_float((uint32_t)hb << 16));
                break;
            }
        }
    }
    if (bad) atomicOr(flags, bad);
}

}  // namespace

cudaError_t launch_dense_prepare(const void* src, int f64, int64_t n, int64_t r0, int64_t nr,
                                 int64_t Np, int layout, void* hi, void* lo, uint32_t* flags,
                                 cudaStream_t st) {
    const int64_t total = nr * n;
    if (total <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    dense_prepare_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, f64, n, r0, nr, Np, layout, hi, lo,
                                                           flags);
    return cudaGetLastError();
}

}  // namespace fth
