// fth_dense_step_noalloc: one dense FP32 fused launch (force, then the element-wise
// GLE step) for callers that cannot allocate device memory.
//
// Who needs it: code that runs where device allocation is not available or not
// allowed -- a plugin whose host framework owns every byte of device memory through
// its own pool, a real-time loop that must never enter the allocator, or an embedded
// caller that only hands the library pointers it already owns.  The regular entry
// points take one caller-provided workspace; this one takes no workspace at all: the
// intermediate force M q lives in a fixed static device array owned by the library.
//
// The paper has no counterpart: this is an allocation policy of the library only.
#include <mutex>

#include "fth.h"
#include "fth_internal.h"

namespace fth {
namespace {

// Scratch for M q: at most kNoallocScratch floats (16 MiB), [n][ldr] row-major.  It is
// one array per device for the whole process (every GPU that loads the library keeps
// it until exit) and every call shares it.
constexpr int64_t kNoallocScratch = int64_t(1) << 22;
static __device__ __align__(256) float g_noalloc_mq[kNoallocScratch];
// The element-wise step tiles replicas by 32 on the grid's y dimension (<= 65535).
constexpr int64_t kNoallocMaxLdr = int64_t(65535) * 32;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_mq_ptr[kMaxDevices] = {};

// MQ[i][r] = sum_k M[i][k] q[k][r] for i < n, r < ldr (every entry written), with
// bounds checks on every load: 64 x 64 tiles, BK 16, 256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256)
noalloc_force_kernel(const float* __restrict__ M, int64_t ldm, const float* __restrict__ q,
                     int64_t ldr, float* __restrict__ MQ, int n) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float As[BK][BM];
    __shared__ float Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    // replica tiles on x (up to 2^31 - 1 blocks), row tiles on y (n <= 2^22 rows)
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < n; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 256) {
            const int rr = e / BK, kk = e % BK;
            const int gi = row0 + rr, gk = k0 + kk;
            As[kk][rr] = (gi < n && gk < n) ? M[(int64_t)gi * ldm + gk] : 0.f;
        }
        for (int e = tid; e < BK * BN; e += 256) {
            const int kk = e / BN, cc = e % BN;
            const int gk = k0 + kk, gc = col0 + cc;
            Bs[kk][cc] = (gk < n && gc < ldr) ? q[(int64_t)gk * ldr + gc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) a[x] = As[kk][ty * 4 + x];
#pragma unroll
            for (int y = 0; y < 4; ++y) b[y] = Bs[kk][tx * 4 + y];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gi = row0 + ty * 4 + x, gc = col0 + tx * 4 + y;
            if (gi < n && gc < ldr) MQ[(int64_t)gi * ldr + gc] = acc[x][y];
        }
}

// Device address of the scratch array on the current device (set up once per device).
fth_status scratch_for_current_device(float** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return FTH_E_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_mq_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_mq) != cudaSuccess || !ptr) return FTH_E_CUDA;
        g_mq_ptr[dev] = static_cast<float*>(ptr);
    }
    *out = g_mq_ptr[dev];
    return FTH_OK;
}

}  // namespace
}  // namespace fth

extern "C" fth_status fth_dense_step_noalloc(const float* M, int64_t n, int64_t ldm, float* q,
                                             float* p, float* s, int64_t replicas, int64_t ldr,
                                             int s_aux, const double* T, const double* S,
                                             double dt, uint64_t seed, uint32_t kappa, int mode,
                                             float* sample, void* stream) {
    using namespace fth;
    if (!M || !q || !p || (s_aux > 0 && !s) || !T || !S) return FTH_E_INVALID_ARG;
    if (n < 1 || ldm < n || replicas < 1 || ldr < replicas || (ldr % 4) != 0) return FTH_E_INVALID_ARG;
    if (s_aux < 0 || s_aux > 4 || !(dt > 0.0) || (mode != 0 && mode != 1)) return FTH_E_INVALID_ARG;
    // n * ldr floats must fit the static scratch (divide first, so absurd sizes cannot
    // overflow), and the element-wise step's grid takes at most kNoallocMaxLdr replicas
    if (ldr > kNoallocMaxLdr || ldr > kNoallocScratch / n) return FTH_E_UNSUPPORTED;
    const uintptr_t mis = reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(p) |
                          reinterpret_cast<uintptr_t>(s) | reinterpret_cast<uintptr_t>(sample);
    if (mis & 15u) return FTH_E_INVALID_ARG;                  // float4 state access
    float* mq = nullptr;
    fth_status st = scratch_for_current_device(&mq);
    if (st != FTH_OK) return st;

    const int ns = s_aux + 1;
    GleF32 g{};
    fill_gle_constants(ns, T, S, &g, nullptr);   // D = T - I, S, joint factor
    g.dt = (float)dt;
    g.hdt = (float)(0.5 * dt);
    g.key0 = (uint32_t)seed;
    g.key1 = (uint32_t)(seed >> 32);
    g.roff = 0;
    set_round_keys(g);
    cudaStream_t strm = static_cast<cudaStream_t>(stream);

    dim3 grid((unsigned)((ldr + 63) / 64), (unsigned)((n + 63) / 64));
    noalloc_force_kernel<<<grid, 256, 0, strm>>>(M, ldm, q, ldr, mq, (int)n);
    if (cudaGetLastError() != cudaSuccess) return FTH_E_CUDA;
    const int flags = mode == 1 ? kDoStart : (kDoEnd | kDoStart | (sample ? kDoSample : 0));
    if (launch_dense_gle(ns, g, n, replicas, ldr, mq, 1, q, p, s, kappa, flags, FTH_OBS_P, sample,
                         ldr, 0, kOpNone, nullptr, nullptr, n, strm) != cudaSuccess)
        return FTH_E_CUDA;
    return FTH_OK;
}
