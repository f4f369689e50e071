// Host runtime of libfth.so: the C ABI of include/fth.h.
//
// fth_create validates the problem, builds the O half-step constants in FP64
// (T = exp(-A_p dt/2), S S^T = C_p - T C_p T^T, Eq. 4 and the cited GLE velocity
// Verlet scheme), carves the caller's device workspace and uploads M.  fth_run
// enqueues, per step, the force (Eq. 5) and the fused GLE step (Eq. 2) on the
// caller's stream, staging one sample per step, and per `stack` samples one
// accumulation pass of the tracked <x_i x_j> (Eq. 6), per `block` samples one FP64
// block flush (the paper's block averaging of the 2A accumulators).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "fth.h"
#include "fth_internal.h"

using namespace fth;

namespace {

thread_local std::string g_thread_error;

constexpr int64_t kGatherMax = int64_t(1) << 20;   // elements per fth_elements gather pass

int64_t round_up(int64_t x, int64_t m) { return ((x + m - 1) / m) * m; }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

enum Path { kPathDense32 = 0, kPathCsr = 1, kPathDense64 = 2 };

// Problem geometry and workspace offsets, computed identically by
// fth_workspace_size and fth_create.
struct Layout {
    Path path;
    int ns;
    int precision, track;
    int64_t N, R, Rp, Np, nnz, stack, ps_ld, ntracked, count, nbt, gcap;
    size_t off_M = 0, off_Mlo = 0, off_rowptr = 0, off_col = 0, off_val = 0;
    size_t off_q0 = 0, off_q1 = 0, off_p = 0, off_s = 0, off_MQ = 0, off_ophi = 0, off_oplo = 0;
    size_t off_ps = 0, off_ps1 = 0, off_pairs = 0, off_partial = 0, off_mean = 0, off_m2 = 0;
    size_t off_prow = 0, off_pcol = 0, off_pe = 0;   // pairs grouped by row (FP32 list paths)
    size_t off_gidx = 0, off_gout = 0, off_err = 0;
    size_t off_xi = 0;       // FP64 path: normals of one segment
    int64_t xi_chunk = 0;    // kick indices per segment that the buffer holds
    size_t total = 0;
};

// The tensor-core paths accumulate every element from a BF16 stack of samples.
bool bf16_stack(const Layout& L) {
    return L.path == kPathDense32 && L.track == FTH_TRACK_ALL &&
           (L.precision == FTH_PREC_TF32 || L.precision == FTH_PREC_BF16X3);
}

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off = align256(off + std::max<size_t>(bytes, 1));
        return o;
    }
};

fth_status fail(std::string* where, fth_status st, const std::string& msg) {
    if (where) *where = msg;
    else g_thread_error = msg;
    return st;
}

// ------------------------------------------------------------------ FP64 propagator
// exp(X) by scaling and squaring with a degree-20 Taylor polynomial: X is scaled by
// 2^-j until its 1-norm is at most 1/2, where the truncated series error is below
// 0.5^21 / 21! (far under FP64 round-off), then squared j times.
void mat_mul(int n, const double* a, const double* b, double* c) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += a[i * n + k] * b[k * n + j];
            c[i * n + j] = acc;
        }
}

void mat_exp(int n, const double* x, double* out) {
    double norm = 0.0;
    for (int j = 0; j < n; ++j) {
        double col = 0.0;
        for (int i = 0; i < n; ++i) col += std::fabs(x[i * n + j]);
        norm = std::max(norm, col);
    }
    int sq = 0;
    double scale = 1.0;
    while (norm * scale > 0.5) {
        scale *= 0.5;
        ++sq;
    }
    std::vector<double> xs(n * n), term(n * n), tmp(n * n);
    for (int k = 0; k < n * n; ++k) xs[k] = x[k] * scale;
    for (int k = 0; k < n * n; ++k) out[k] = (k % (n + 1) == 0) ? 1.0 : 0.0;
    for (int k = 0; k < n * n; ++k) term[k] = out[k];
    for (int d = 1; d <= 20; ++d) {
        mat_mul(n, term.data(), xs.data(), tmp.data());
        for (int k = 0; k < n * n; ++k) {
            term[k] = tmp[k] / d;
            out[k] += term[k];
        }
    }
    for (int s = 0; s < sq; ++s) {
        mat_mul(n, out, out, tmp.data());
        std::copy(tmp.begin(), tmp.end(), out);
    }
}

// Lower-triangular L with L L^T = a (symmetric PSD); a pivot at or below
// 1e-14 * max diag is an exact zero and its column is left zero.
void chol_psd(int n, const double* a_in, double* L) {
    std::vector<double> a(a_in, a_in + n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) a[i * n + j] = a[j * n + i] = 0.5 * (a[i * n + j] + a[j * n + i]);
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) dmax = std::max(dmax, a[i * n + i]);
    const double tol = 1e-14 * dmax;
    std::fill(L, L + n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > tol)) continue;
        const double ljj = std::sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = a[i * n + j];
            for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = v / ljj;
        }
    }
}

}  // namespace

// The sample (end of step kappa - 1) observes p between the two O half-steps of a fused
// launch.  From the state v after the end-of-step kick, the sample is (T v)_0 + x and
// the next mid-step state T T v + y, with x = e_0^T S xi1 and y = T S xi1 + S xi2 for
// independent xi1, xi2.  (x, y) is Gaussian with covariance
//   [[C1_00, (T C1 e_0)^T], [T C1 e_0, T C1 T^T + C1]],  C1 = S S^T,
// so L = chol of it draws both half-steps from ns + 1 normals: the same Markov chain.
void fth::fill_gle_constants(int ns, const double* T, const double* S, GleF32* g32, GleF64* g64) {
    const int m = ns + 1;
    std::vector<double> C1(ns * ns, 0.0), TC1(ns * ns, 0.0), sig(m * m, 0.0), L(m * m, 0.0);
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j)
            for (int k = 0; k < ns; ++k) C1[i * ns + j] += S[i * ns + k] * S[j * ns + k];
    mat_mul(ns, T, C1.data(), TC1.data());
    sig[0] = C1[0];
    for (int a = 0; a < ns; ++a) sig[(a + 1) * m] = sig[a + 1] = TC1[a * ns];
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b) {
            double tct = 0.0;
            for (int k = 0; k < ns; ++k) tct += TC1[a * ns + k] * T[b * ns + k];
            sig[(a + 1) * m + b + 1] = tct + C1[a * ns + b];
        }
    chol_psd(m, sig.data(), L.data());
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b) {
            const double d = T[a * ns + b] - (a == b ? 1.0 : 0.0);
            double t2 = 0.0;
            for (int k = 0; k < ns; ++k) t2 += T[a * ns + k] * T[k * ns + b];
            const double d2 = t2 - (a == b ? 1.0 : 0.0);
            if (g32) {
                g32->T[a * kMaxNs + b] = (float)d;
                g32->S[a * kMaxNs + b] = (float)S[a * ns + b];
                g32->D2[a * kMaxNs + b] = (float)d2;
            }
            if (g64) {
                g64->T[a * kMaxNs + b] = d;
                g64->S[a * kMaxNs + b] = S[a * ns + b];
                g64->D2[a * kMaxNs + b] = d2;
            }
        }
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            if (g32) g32->L[a * kMaxNs1 + b] = (float)L[a * m + b];
            if (g64) g64->L[a * kMaxNs1 + b] = L[a * m + b];
        }
}

namespace {

fth_status propagator(const fth_gle* gle, double dt, double* T, double* S, std::string* msg) {
    if (!gle) return fail(msg, FTH_E_INVALID_ARG, "gle is NULL");
    const int ns = gle->s + 1;
    if (gle->s < 0 || ns > kMaxNs) return fail(msg, FTH_E_UNSUPPORTED, "s must be in [0, 4]");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(msg, FTH_E_INVALID_ARG, "dt must be > 0");
    std::vector<double> x(ns * ns), tct(ns * ns), tmp(ns * ns), tt(ns * ns);
    for (int k = 0; k < ns * ns; ++k) {
        if (!std::isfinite(gle->a_p[k]) || !std::isfinite(gle->c_p[k]))
            return fail(msg, FTH_E_INVALID_ARG, "A_p / C_p not finite");
        x[k] = -0.5 * dt * gle->a_p[k];
    }
    mat_exp(ns, x.data(), T);
    // C_p - T C_p T^T
    mat_mul(ns, T, gle->c_p, tmp.data());
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) tt[i * ns + j] = T[j * ns + i];
    mat_mul(ns, tmp.data(), tt.data(), tct.data());
    for (int k = 0; k < ns * ns; ++k) tct[k] = gle->c_p[k] - tct[k];
    for (int i = 0; i < ns; ++i)
        if (tct[i * ns + i] < -1e-12 * std::max(1.0, std::fabs(gle->c_p[i * ns + i])))
            return fail(msg, FTH_E_INVALID_ARG,
                        "C_p - T C_p T^T is not positive semi-definite (invalid GLE)");
    chol_psd(ns, tct.data(), S);
    for (int k = 0; k < ns * ns; ++k)
        if (!std::isfinite(T[k]) || !std::isfinite(S[k]))
            return fail(msg, FTH_E_INVALID_ARG, "propagator not finite");
    return FTH_OK;
}

// ------------------------------------------------------------------ validation + layout
fth_status plan(const fth_matrix* M, const fth_gle* gle, const fth_options* o, Layout* L,
                std::string* msg) {
    if (!M || !gle || !o || !L) return fail(msg, FTH_E_INVALID_ARG, "NULL argument");
    if (M->n < 1 || M->n > (1ll << 30)) return fail(msg, FTH_E_INVALID_ARG, "n out of range");
    if (!M->values) return fail(msg, FTH_E_INVALID_ARG, "matrix values are NULL");
    if (M->dtype != FTH_F32 && M->dtype != FTH_F64) return fail(msg, FTH_E_INVALID_ARG, "bad dtype");
    if (M->kind != FTH_DENSE && M->kind != FTH_CSR) return fail(msg, FTH_E_INVALID_ARG, "bad kind");
    if (gle->s < 0 || gle->s > 4) return fail(msg, FTH_E_UNSUPPORTED, "s must be in [0, 4]");
    if (o->replicas < 1 || o->replicas > (1ll << 24))
        return fail(msg, FTH_E_INVALID_ARG, "replicas out of range");
    if (!(o->dt > 0.0)) return fail(msg, FTH_E_INVALID_ARG, "dt must be > 0");
    if (o->block < 1 || o->burnin < 0) return fail(msg, FTH_E_INVALID_ARG, "block >= 1, burnin >= 0");
    if (o->observable != FTH_OBS_P && o->observable != FTH_OBS_Q)
        return fail(msg, FTH_E_INVALID_ARG, "bad observable");
    if (o->precision < FTH_PREC_FP32 || o->precision > FTH_PREC_FP64)
        return fail(msg, FTH_E_INVALID_ARG, "bad precision");
    if (o->track < FTH_TRACK_LIST || o->track > FTH_TRACK_ALL)
        return fail(msg, FTH_E_INVALID_ARG, "bad track");
    if (o->track == FTH_TRACK_LIST && (o->npairs < 0 || (o->npairs > 0 && !o->pairs)))
        return fail(msg, FTH_E_INVALID_ARG, "pairs");
    if (o->stack < 0) return fail(msg, FTH_E_INVALID_ARG, "stack must be >= 0");
    if (o->replica_offset < 0 || o->replica_offset + o->replicas > (1ll << 32))
        return fail(msg, FTH_E_INVALID_ARG, "replica_offset + replicas must fit in 32 bits");

    *L = Layout();
    L->ns = gle->s + 1;
    L->N = M->n;
    L->R = o->replicas;
    L->precision = o->precision;
    L->track = o->track;
    const bool tc = o->precision == FTH_PREC_TF32 || o->precision == FTH_PREC_BF16X3;
    if (M->kind == FTH_CSR) {
        if (o->precision != FTH_PREC_FP32)
            return fail(msg, FTH_E_UNSUPPORTED, "CSR matrices use the FP32 SpMM path");
        if (o->track == FTH_TRACK_ALL)
            return fail(msg, FTH_E_UNSUPPORTED, "track ALL is for dense matrices");
        if (!M->rowptr || !M->colind || M->nnz < 0)
            return fail(msg, FTH_E_INVALID_ARG, "CSR arrays");
        L->path = kPathCsr;
        L->nnz = M->nnz;
        L->Np = L->N;
    } else if (o->precision == FTH_PREC_FP64) {
        if (M->n > 1024) return fail(msg, FTH_E_UNSUPPORTED, "FP64 path supports n <= 1024");
        L->path = kPathDense64;
        L->Np = round_up(L->N, 32);
    } else {
        L->path = kPathDense32;
        L->Np = round_up(L->N, kTile);
    }
    // replicas padded to a float4 (element-wise kernels); the tensor-core paths pad to
    // the 64-wide force tile so TMA boxes never exceed the tensor and every staged
    // SYRK slice of 32 columns holds whole samples
    L->Rp = round_up(L->R, tc ? 64 : 4);

    // tracked elements
    int64_t ntracked = 0;
    if (L->path == kPathDense64) {
        if (o->track == FTH_TRACK_LIST) ntracked = o->npairs;
        else if (o->track == FTH_TRACK_DIAG) ntracked = L->N;
        else ntracked = L->N * (L->N + 1) / 2;
    } else if (o->track == FTH_TRACK_LIST) {
        ntracked = o->npairs;
    } else if (o->track == FTH_TRACK_DIAG) {
        ntracked = L->N;
    }
    L->ntracked = ntracked;
    const bool all32 = L->path == kPathDense32 && o->track == FTH_TRACK_ALL;
    L->nbt = all32 ? L->Np / kTile : 0;
    L->count = all32 ? (L->nbt * (L->nbt + 1) / 2) * kTile * kTile : ntracked;
    if (o->track == FTH_TRACK_LIST && o->pairs) {
        for (int64_t e = 0; e < o->npairs; ++e) {
            const int64_t i = o->pairs[2 * e], j = o->pairs[2 * e + 1];
            if (i < 0 || j < 0 || i >= L->N || j >= L->N)
                return fail(msg, FTH_E_INVALID_ARG, "pair index out of range");
        }
    }
    if (L->path != kPathDense64) {
        // auto: 2048 FP32 or 4096 BF16 staged columns (8 KiB per row) per pass
        const int64_t cols = bf16_stack(*L) ? 4096 : 2048;
        L->stack = o->stack > 0 ? o->stack
                                : (all32 ? std::max<int64_t>(1, cols / L->Rp) : 4);
        L->ps_ld = L->stack * L->Rp;
    }

    // workspace carving
    Carve c;
    const int64_t N = L->N, Np = L->Np, Rp = L->Rp;
    const int nsub = L->ns - 1;
    if (L->path == kPathDense32) {
        const size_t esz = o->precision == FTH_PREC_BF16X3 ? 2 : 4;
        L->off_M = c.take((size_t)Np * Np * esz);
        if (o->precision == FTH_PREC_BF16X3) L->off_Mlo = c.take((size_t)Np * Np * esz);
        L->off_q0 = c.take((size_t)Np * Rp * 4);
        L->off_p = c.take((size_t)Np * Rp * 4);
        L->off_s = c.take((size_t)std::max(nsub, 1) * Np * Rp * 4);
        const int planes = tc ? 1 : sgemm_force_planes(Rp);      // FP32: K shares summed later
        L->off_MQ = c.take((size_t)planes * Np * Rp * 4);
        if (tc) {
            L->off_ophi = c.take((size_t)Rp * Np * esz);
            if (o->precision == FTH_PREC_BF16X3) L->off_oplo = c.take((size_t)Rp * Np * esz);
        }
        const size_t ps_esz = bf16_stack(*L) ? 2 : 4;
        L->off_ps = c.take((size_t)Np * L->ps_ld * ps_esz);
        L->off_ps1 = c.take((size_t)Np * L->ps_ld * ps_esz);
    } else if (L->path == kPathCsr) {
        L->off_rowptr = c.take((size_t)(N + 1) * 4);
        L->off_col = c.take((size_t)std::max<int64_t>(L->nnz, 1) * 4);
        L->off_val = c.take((size_t)std::max<int64_t>(L->nnz, 1) * 4);
        L->off_q0 = c.take((size_t)N * Rp * 4);
        L->off_q1 = c.take((size_t)N * Rp * 4);
        L->off_p = c.take((size_t)N * Rp * 4);
        L->off_s = c.take((size_t)std::max(nsub, 1) * N * Rp * 4);
        L->off_ps = c.take((size_t)N * L->ps_ld * 4);
        L->off_ps1 = c.take((size_t)N * L->ps_ld * 4);
    } else {
        L->off_M = c.take((size_t)N * Np * 8);
        L->off_q0 = c.take((size_t)L->R * Np * 8);
        L->off_p = c.take((size_t)L->R * Np * 8);
        L->off_s = c.take((size_t)std::max(nsub, 1) * L->R * Np * 8);
        // normals generated ahead: up to 4096 kick indices, at most ~64 MiB
        const size_t per = (size_t)L->R * (L->ns + 1) * Np * 8;
        L->xi_chunk = std::max<int64_t>(2, std::min<int64_t>(4096, (int64_t)((size_t(64) << 20) / per)));
        L->off_xi = c.take(per * (size_t)L->xi_chunk);
    }
    L->off_pairs = c.take((size_t)std::max<int64_t>(ntracked, 1) * 2 * 4);
    if (L->path != kPathDense64 && o->track != FTH_TRACK_ALL) {
        L->off_prow = c.take((size_t)(L->N + 1) * 4);
        L->off_pcol = c.take((size_t)std::max<int64_t>(ntracked, 1) * 4);
        L->off_pe = c.take((size_t)std::max<int64_t>(ntracked, 1) * 4);
    }
    if (L->path == kPathDense64) L->off_partial = c.take((size_t)std::max<int64_t>(L->count, 1) * L->R * 8);
    else L->off_partial = c.take((size_t)std::max<int64_t>(L->count, 1) * 4);
    L->off_mean = c.take((size_t)std::max<int64_t>(L->count, 1) * 8);
    L->off_m2 = c.take((size_t)std::max<int64_t>(L->count, 1) * 8);
    // gather capacity: every element a request can name (tile-packed count when all are
    // tracked on the dense FP32 path, where ntracked is 0), at most kGatherMax per pass
    L->gcap = std::max<int64_t>(1, std::min<int64_t>(std::max(L->ntracked, L->count), kGatherMax));
    L->off_gidx = c.take((size_t)L->gcap * 8);
    L->off_gout = c.take((size_t)L->gcap * 3 * 8);
    L->off_err = c.take(256);
    L->total = c.off;
    return FTH_OK;
}

inline uint16_t bf16_rne(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);  // inf / nan
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
inline float bf16_to_f(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

inline float tf32_rna(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) != 0x7F800000u) {
        u += 0x1000u;
        u &= ~0x1FFFu;
    }
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

}  // namespace

// ======================================================================== context
struct fth_ctx {
    Layout L;
    cudaStream_t stream = nullptr;
    int observable = 0;
    int64_t burnin = 0, block = 1;
    uint64_t seed = 0;
    double dt = 0;
    double T[kMaxNs * kMaxNs] = {}, S[kMaxNs * kMaxNs] = {};
    GleF32 g32{};
    GleF64 g64{};
    uint8_t* ws = nullptr;
    size_t ws_bytes = 0;
    // device pointers
    void* M = nullptr;
    void* Mlo = nullptr;
    int32_t *rowptr = nullptr, *col = nullptr;
    float* val = nullptr;
    void* q[2] = {nullptr, nullptr};
    void *p = nullptr, *s = nullptr;
    float* MQ = nullptr;
    void *ophi = nullptr, *oplo = nullptr;
    float* ps = nullptr;          // sample stack being filled (one of psb)
    float* psb[2] = {nullptr, nullptr};
    int psi = 0;                  // index of the stack being filled
    // accumulation passes and block flushes other than the tensor-core pass over all
    // elements run on a side stream, overlapping the next steps; events order them
    // against the caller's stream (acc_stream)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_filled[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_join = nullptr;
    bool free_pending[2] = {false, false};
    bool side_used = false;
    int32_t* pairs = nullptr;
    void* partial = nullptr;
    double *mean = nullptr, *m2 = nullptr;
    int64_t* gidx = nullptr;
    double* gout = nullptr;
    uint32_t* err = nullptr;
    TcForce* tcf = nullptr;
    TcSyrk* tcs = nullptr;
    TcSyrk* tcs1 = nullptr;
    // host-side bookkeeping
    std::vector<int32_t> reg_pairs;                        // registered pairs (i <= j), in order
    std::unordered_map<uint64_t, int64_t> pair_index;      // built on the first out-of-order lookup
    int32_t* prow = nullptr;   // tracked pairs grouped by first index (device)
    int32_t* pcol = nullptr;
    int32_t* pe = nullptr;
    // linear functionals (device storage owned by the caller)
    struct Functional {
        int64_t* idx;
        double* w;
        double* acc;        // [0] block value being formed, [1] Welford mean, [2] M2
        int64_t nterms;
        std::vector<int64_t> pairs;
        std::vector<double> weights;
    };
    std::vector<Functional> funcs;
    int64_t t = 0, nsamp = 0, accumulated = 0, inblock = 0, nfill = 0, nblocks = 0, launches = 0;
    int primed = 0, cur = 0;
    std::string last_error;
    // opt-in per-launch event timing
    bool prof = false;
    struct ProfRec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[FTH_K_CLASSES] = {};
    int64_t prof_n[FTH_K_CLASSES] = {};
};

namespace {

uint64_t pair_key(int64_t i, int64_t j) {
    if (i > j) std::swap(i, j);
    return ((uint64_t)i << 32) | (uint64_t)j;
}

fth_status cuda_fail(fth_ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (c) c->last_error = m;
    else g_thread_error = m;
    return FTH_E_CUDA;
}

#define FTH_CK(call, what)                                 \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

cudaEvent_t prof_event(fth_ctx* c) {
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one kernel launch with an event pair when profiling is on.
struct ProfScope {
    fth_ctx* c;
    bool on;
    cudaStream_t st;
    size_t idx = 0;
    ProfScope(fth_ctx* ctx, int cls, cudaStream_t s = nullptr)
        : c(ctx), on(ctx->prof), st(s ? s : ctx->stream) {
        if (!on) return;
        fth_ctx::ProfRec r{cls, prof_event(c), prof_event(c)};
        cudaEventRecord(r.a, st);
        idx = c->prof_recs.size();
        c->prof_recs.push_back(r);
    }
    ~ProfScope() {
        if (on) cudaEventRecord(c->prof_recs[idx].b, st);
    }
};

bool is_tc(const fth_ctx* c) {
    return c->L.path == kPathDense32 &&
           (c->L.precision == FTH_PREC_TF32 || c->L.precision == FTH_PREC_BF16X3);
}

fth_status force(fth_ctx* c) {
    const Layout& L = c->L;
    ProfScope ps(c, is_tc(c) ? FTH_K_FORCE_TC : FTH_K_FORCE_FP32);
    if (is_tc(c)) {
        FTH_CK(tc_force_run(c->tcf, c->MQ, L.Rp, c->err, c->stream), "tc force");
    } else {
        FTH_CK(launch_sgemm_force(static_cast<const float*>(c->M), L.Np,
                                  static_cast<const float*>(c->q[0]), L.Rp, c->MQ, L.N, c->stream),
               "sgemm force");
    }
    ++c->launches;
    return FTH_OK;
}

// Before the first sample of a stack is written: the pass that read this stack two
// batches ago must be finished.
fth_status claim_stack(fth_ctx* c) {
    if (c->free_pending[c->psi]) {
        FTH_CK(cudaStreamWaitEvent(c->stream, c->ev_free[c->psi], 0), "wait stack");
        c->free_pending[c->psi] = false;
    }
    c->ps = c->psb[c->psi];
    return FTH_OK;
}

// The stream of the accumulation passes and block flushes.  The tensor-core pass over
// all elements runs in line on the caller's stream: beside the next steps its CTAs held
// SMs the force needed, which cost more than the pass itself.  The other passes run on
// the side stream, beside the next steps.
cudaStream_t acc_stream(const fth_ctx* c) {
    return c->L.track == FTH_TRACK_ALL && is_tc(c) ? c->stream : c->side;
}

// One accumulation pass over the filled stack; the other stack takes the next samples
// meanwhile.
fth_status accumulate(fth_ctx* c) {
    const Layout& L = c->L;
    if (c->nfill == 0) return FTH_OK;
    const int64_t ncols = c->nfill * L.Rp;
    const int b = c->psi;
    const cudaStream_t as = acc_stream(c);
    if (as != c->stream) {
        FTH_CK(cudaEventRecord(c->ev_filled[b], c->stream), "record filled");
        FTH_CK(cudaStreamWaitEvent(as, c->ev_filled[b], 0), "side wait");
        c->side_used = true;
    }
    {
        ProfScope ps(c, L.track == FTH_TRACK_ALL ? (is_tc(c) ? FTH_K_SYRK_TC : FTH_K_SYRK_FP32)
                                                 : FTH_K_PAIR_ACCUM,
                     as);
        if (L.track == FTH_TRACK_ALL) {
            if (is_tc(c)) {
                FTH_CK(tc_syrk_run(b ? c->tcs1 : c->tcs, ncols, static_cast<float*>(c->partial),
                                   c->err, as),
                       "tc syrk");
            } else {
                FTH_CK(launch_syrk_fp32(c->psb[b], L.ps_ld, ncols, L.Np,
                                        static_cast<float*>(c->partial), as),
                       "syrk");
            }
        } else if (c->prow && pair_accum_rows_supported(ncols)) {
            FTH_CK(launch_pair_accum_rows(c->psb[b], L.ps_ld, ncols, c->prow, c->pcol, c->pe, L.N,
                                          static_cast<float*>(c->partial), as),
                   "pair accumulate (rows)");
        } else {
            FTH_CK(launch_pair_accum(c->psb[b], L.ps_ld, ncols, c->pairs, L.ntracked,
                                     static_cast<float*>(c->partial), as),
                   "pair accumulate");
        }
    }
    FTH_CK(cudaEventRecord(c->ev_free[b], as), "record free");
    c->free_pending[b] = true;
    ++c->launches;
    c->nfill = 0;
    c->psi ^= 1;
    return FTH_OK;
}

// The caller's stream waits for everything queued on the side stream.
fth_status join_side(fth_ctx* c) {
    if (!c->side_used) return FTH_OK;
    FTH_CK(cudaEventRecord(c->ev_join, c->side), "record join");
    FTH_CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join");
    c->side_used = false;
    return FTH_OK;
}

fth_status flush(fth_ctx* c) {
    const Layout& L = c->L;
    const double inv = 1.0 / ((double)c->block * (double)L.R);
    const double nb = (double)(c->nblocks + 1);
    // functionals first: they read the block's partial sums before the flush clears them
    for (auto& f : c->funcs) {
        const bool p64 = L.path == kPathDense64;
        cudaStream_t st = p64 ? c->stream : acc_stream(c);
        FTH_CK(launch_functional_block(p64 ? nullptr : static_cast<const float*>(c->partial),
                                       p64 ? static_cast<const double*>(c->partial) : nullptr,
                                       L.R, L.count, f.idx, f.w, f.nterms, inv, nb, f.acc, c->err,
                                       st),
               "functional");
        c->launches += 2;
    }
    if (L.path == kPathDense64) {
        ProfScope ps(c, FTH_K_FLUSH);
        FTH_CK(launch_flush64(static_cast<double*>(c->partial), L.R, L.count, c->mean, c->m2,
                              L.count, inv, nb, c->err, c->stream),
               "flush64");
    } else {
        // after the block's last accumulation pass, on the same stream
        const cudaStream_t as = acc_stream(c);
        ProfScope ps(c, FTH_K_FLUSH, as);
        FTH_CK(launch_flush(static_cast<float*>(c->partial), c->mean, c->m2, L.count, inv, nb,
                            c->err, as),
               "flush");
        if (as != c->stream) c->side_used = true;
    }
    ++c->launches;
    ++c->nblocks;
    c->inblock = 0;
    return FTH_OK;
}

// The tensor-core forces arrive as one plane (their K shares are reduced on chip or in
// L2); the FP32 force writes one plane per K share.
int mq_planes(const fth_ctx* c) { return is_tc(c) ? 1 : sgemm_force_planes(c->L.Rp); }

// kZeroMQ when the force adds its partial sums into MQ (the element-wise step zeroes it).
int zero_mq(const fth_ctx* c) { return c->tcf && tc_force_accumulates(c->tcf) ? kZeroMQ : 0; }

void op_ptrs(fth_ctx* c, int& kind, void*& hi, void*& lo) {
    kind = kOpNone;
    hi = lo = nullptr;
    if (c->L.path != kPathDense32) return;
    if (c->L.precision == FTH_PREC_TF32) kind = kOpTf32;
    if (c->L.precision == FTH_PREC_BF16X3) kind = kOpBf16x2;
    hi = c->ophi;
    lo = c->oplo;
}

fth_status run_dense32(fth_ctx* c, int64_t steps) {
    const Layout& L = c->L;
    int opk;
    void *hi, *lo;
    op_ptrs(c, opk, hi, lo);
    float* q = static_cast<float*>(c->q[0]);
    float* p = static_cast<float*>(c->p);
    float* s = static_cast<float*>(c->s);
    if (!c->primed) {
        fth_status st = force(c);
        if (st != FTH_OK) return st;
        {
            ProfScope ps(c, FTH_K_GLE_DENSE);
            FTH_CK(launch_dense_gle(L.ns, c->g32, L.N, L.R, L.Rp, c->MQ, mq_planes(c), q, p, s,
                                    (uint32_t)c->t, kDoStart | zero_mq(c), c->observable, c->ps,
                                    L.ps_ld, 0, opk, hi, lo, L.Np, c->stream),
                   "gle prologue");
        }
        ++c->launches;
        c->primed = 1;
    }
    for (int64_t k = 0; k < steps; ++k) {
        const uint32_t kappa = (uint32_t)(c->t + 1);
        fth_status st = force(c);
        if (st != FTH_OK) return st;
        const bool take = c->nsamp >= c->burnin;
        // the tcgen05 accumulation pass reads a BF16 stack (samples rounded to nearest)
        const int flags = kDoEnd | kDoStart | (take ? kDoSample : 0) |
                          (take && bf16_stack(L) ? kSampleBf16 : 0) | zero_mq(c);
        if (take && c->nfill == 0) {
            st = claim_stack(c);
            if (st != FTH_OK) return st;
        }
        {
            ProfScope ps(c, FTH_K_GLE_DENSE);
            FTH_CK(launch_dense_gle(L.ns, c->g32, L.N, L.R, L.Rp, c->MQ, mq_planes(c), q, p, s,
                                    kappa, flags, c->observable, c->ps, L.ps_ld, c->nfill, opk,
                                    hi, lo, L.Np, c->stream),
                   "gle step");
        }
        ++c->launches;
        ++c->t;
        ++c->nsamp;
        if (take) {
            ++c->nfill;
            ++c->inblock;
            ++c->accumulated;
            if (c->nfill == L.stack || c->inblock == c->block) {
                st = accumulate(c);
                if (st != FTH_OK) return st;
            }
            if (c->inblock == c->block) {
                st = flush(c);
                if (st != FTH_OK) return st;
            }
        }
    }
    fth_status st = accumulate(c);
    if (st != FTH_OK) return st;
    return join_side(c);
}

fth_status run_csr(fth_ctx* c, int64_t steps) {
    const Layout& L = c->L;
    float* p = static_cast<float*>(c->p);
    float* s = static_cast<float*>(c->s);
    auto launch = [&](int flags, uint32_t kappa) -> fth_status {
        float* qin = static_cast<float*>(c->q[c->cur]);
        float* qout = static_cast<float*>(c->q[c->cur ^ 1]);
        ProfScope ps(c, FTH_K_CSR_STEP);
        FTH_CK(launch_csr_step(L.ns, c->g32, L.N, L.R, L.Rp, c->rowptr, c->col, c->val, qin, qout,
                               p, s, kappa, flags, c->observable, c->ps, L.ps_ld, c->nfill,
                               c->stream),
               "csr step");
        ++c->launches;
        c->cur ^= 1;
        return FTH_OK;
    };
    if (!c->primed) {
        fth_status st = launch(kDoStart, (uint32_t)c->t);
        if (st != FTH_OK) return st;
        c->primed = 1;
    }
    for (int64_t k = 0; k < steps; ++k) {
        const bool take = c->nsamp >= c->burnin;
        if (take && c->nfill == 0) {
            fth_status st0 = claim_stack(c);
            if (st0 != FTH_OK) return st0;
        }
        fth_status st = launch(kDoEnd | kDoStart | (take ? kDoSample : 0), (uint32_t)(c->t + 1));
        if (st != FTH_OK) return st;
        ++c->t;
        ++c->nsamp;
        if (take) {
            ++c->nfill;
            ++c->inblock;
            ++c->accumulated;
            if (c->nfill == L.stack || c->inblock == c->block) {
                st = accumulate(c);
                if (st != FTH_OK) return st;
            }
            if (c->inblock == c->block) {
                st = flush(c);
                if (st != FTH_OK) return st;
            }
        }
    }
    fth_status st = accumulate(c);
    if (st != FTH_OK) return st;
    return join_side(c);
}

fth_status run_dense64(fth_ctx* c, int64_t steps) {
    const Layout& L = c->L;
    while (steps > 0 || !c->primed) {
        // one segment: up to the end of the current block (or the burn-in), in one launch
        int64_t seg = steps;
        int64_t acc_from = 0;
        if (c->nsamp < c->burnin) {
            acc_from = c->burnin - c->nsamp;
            seg = std::min(seg, acc_from + (c->block - c->inblock));
        } else {
            seg = std::min(seg, c->block - c->inblock);
        }
        seg = std::min<int64_t>(seg, L.xi_chunk - (c->primed ? 0 : 1));
        const uint32_t kappa0 = (uint32_t)(c->primed ? c->t + 1 : c->t);
        double* xi = reinterpret_cast<double*>(c->ws + L.off_xi);
        {
        ProfScope ps(c, FTH_K_FP64_NOISE);
        FTH_CK(launch_fp64_noise(L.ns, c->g64, L.N, L.Np, L.R, kappa0, seg + (c->primed ? 0 : 1),
                                 c->primed ? 0 : 1, xi, c->stream),
               "fp64 noise");
        }
        ++c->launches;
        {
        ProfScope ps(c, FTH_K_FP64_DENSE);
        FTH_CK(launch_fp64_dense(L.ns, c->g64, L.N, L.Np, L.R, static_cast<const double*>(c->M),
                                 static_cast<double*>(c->q[0]), static_cast<double*>(c->p),
                                 static_cast<double*>(c->s), xi, seg, c->primed,
                                 c->observable, c->pairs, L.ntracked,
                                 static_cast<double*>(c->partial), acc_from, c->stream),
               "fp64 dense");
        }
        ++c->launches;
        c->primed = 1;
        c->t += seg;
        c->nsamp += seg;
        const int64_t took = std::max<int64_t>(0, seg - acc_from);
        c->inblock += took;
        c->accumulated += took;
        steps -= seg;
        if (c->inblock == c->block) {
            fth_status st = flush(c);
            if (st != FTH_OK) return st;
        }
        if (seg == 0 && steps == 0) break;
    }
    return FTH_OK;
}

fth_status upload_state_operand(fth_ctx* c) {
    // refresh the transposed force operand from the FP32 q plane (TC paths)
    const Layout& L = c->L;
    if (!is_tc(c)) return FTH_OK;
    std::vector<float> q((size_t)L.Np * L.Rp);
    FTH_CK(cudaMemcpyAsync(q.data(), c->q[0], q.size() * 4, cudaMemcpyDeviceToHost, c->stream),
           "d2h q");
    FTH_CK(cudaStreamSynchronize(c->stream), "sync");
    if (L.precision == FTH_PREC_TF32) {
        std::vector<float> t((size_t)L.Rp * L.Np, 0.f);
        for (int64_t i = 0; i < L.N; ++i)
            for (int64_t r = 0; r < L.Rp; ++r) t[r * L.Np + i] = tf32_rna(q[i * L.Rp + r]);
        FTH_CK(cudaMemcpyAsync(c->ophi, t.data(), t.size() * 4, cudaMemcpyHostToDevice, c->stream),
               "h2d op");
    } else {
        std::vector<uint16_t> h((size_t)L.Rp * L.Np, 0), l((size_t)L.Rp * L.Np, 0);
        for (int64_t i = 0; i < L.N; ++i)
            for (int64_t r = 0; r < L.Rp; ++r) {
                const float x = q[i * L.Rp + r];
                const uint16_t hb = bf16_rne(x);
                h[r * L.Np + i] = hb;
                l[r * L.Np + i] = bf16_rne(x - bf16_to_f(hb));
            }
        FTH_CK(cudaMemcpyAsync(c->ophi, h.data(), h.size() * 2, cudaMemcpyHostToDevice, c->stream),
               "h2d op hi");
        FTH_CK(cudaMemcpyAsync(c->oplo, l.data(), l.size() * 2, cudaMemcpyHostToDevice, c->stream),
               "h2d op lo");
    }
    FTH_CK(cudaStreamSynchronize(c->stream), "sync");
    return FTH_OK;
}

}  // namespace

// ======================================================================== C ABI
extern "C" {

const char* fth_version(void) { return "fth 0.1 (sm_103a)"; }

const char* fth_last_error(const fth_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : g_thread_error.c_str();
}

fth_status fth_gle_propagator(const fth_gle* gle, double dt, double* T, double* S) {
    if (!T || !S) return fail(nullptr, FTH_E_INVALID_ARG, "NULL output");
    return propagator(gle, dt, T, S, nullptr);
}

fth_status fth_workspace_size(const fth_matrix* M, const fth_gle* gle, const fth_options* opt,
                              size_t* bytes) {
    if (!bytes) return fail(nullptr, FTH_E_INVALID_ARG, "bytes is NULL");
    Layout L;
    fth_status st = plan(M, gle, opt, &L, nullptr);
    if (st != FTH_OK) return st;
    *bytes = L.total;
    return FTH_OK;
}

fth_status fth_create(const fth_matrix* Min, const fth_gle* gle, const fth_options* opt,
                      void* workspace, size_t workspace_bytes, fth_ctx** out) {
    if (!out) return fail(nullptr, FTH_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    Layout L;
    fth_status st = plan(Min, gle, opt, &L, nullptr);
    if (st != FTH_OK) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return fail(nullptr, FTH_E_WORKSPACE, "workspace must be 256-byte aligned device memory");
    if (workspace_bytes < L.total)
        return fail(nullptr, FTH_E_WORKSPACE, "workspace too small: need " + std::to_string(L.total) +
                                                  " bytes");
    fth_ctx* c = new fth_ctx();
    c->L = L;
    c->stream = static_cast<cudaStream_t>(opt->stream);
    c->observable = opt->observable;
    c->burnin = opt->burnin;
    c->block = opt->block;
    c->seed = opt->seed;
    c->dt = opt->dt;
    c->ws = static_cast<uint8_t*>(workspace);
    c->ws_bytes = workspace_bytes;
    st = propagator(gle, opt->dt, c->T, c->S, &c->last_error);
    if (st != FTH_OK) {
        g_thread_error = c->last_error;
        delete c;
        return st;
    }
    fill_gle_constants(L.ns, c->T, c->S, &c->g32, &c->g64);
    c->g32.dt = (float)opt->dt;
    c->g32.hdt = (float)(0.5 * opt->dt);
    c->g64.dt = opt->dt;
    c->g64.hdt = 0.5 * opt->dt;
    c->g32.key0 = c->g64.key0 = (uint32_t)opt->seed;
    c->g32.key1 = c->g64.key1 = (uint32_t)(opt->seed >> 32);
    c->g32.roff = c->g64.roff = (uint32_t)opt->replica_offset;
    set_round_keys(c->g32);

    auto at = [&](size_t off) { return static_cast<void*>(c->ws + off); };
    c->M = at(L.off_M);
    c->Mlo = L.off_Mlo ? at(L.off_Mlo) : nullptr;
    c->q[0] = at(L.off_q0);
    c->q[1] = L.off_q1 ? at(L.off_q1) : nullptr;
    c->p = at(L.off_p);
    c->s = at(L.off_s);
    c->MQ = L.off_MQ ? static_cast<float*>(at(L.off_MQ)) : nullptr;
    c->ophi = L.off_ophi ? at(L.off_ophi) : nullptr;
    c->oplo = L.off_oplo ? at(L.off_oplo) : nullptr;
    c->psb[0] = L.off_ps ? static_cast<float*>(at(L.off_ps)) : nullptr;
    c->psb[1] = L.off_ps1 ? static_cast<float*>(at(L.off_ps1)) : nullptr;
    c->ps = c->psb[0];
    c->pairs = static_cast<int32_t*>(at(L.off_pairs));
    if (L.off_prow) {
        c->prow = static_cast<int32_t*>(at(L.off_prow));
        c->pcol = static_cast<int32_t*>(at(L.off_pcol));
        c->pe = static_cast<int32_t*>(at(L.off_pe));
    }
    c->partial = at(L.off_partial);
    c->mean = static_cast<double*>(at(L.off_mean));
    c->m2 = static_cast<double*>(at(L.off_m2));
    c->gidx = static_cast<int64_t*>(at(L.off_gidx));
    c->gout = static_cast<double*>(at(L.off_gout));
    c->err = static_cast<uint32_t*>(at(L.off_err));
    if (L.path == kPathCsr) {
        c->rowptr = static_cast<int32_t*>(at(L.off_rowptr));
        c->col = static_cast<int32_t*>(at(L.off_col));
        c->val = static_cast<float*>(at(L.off_val));
    }

    auto bail = [&](fth_status s2) {
        g_thread_error = c->last_error;
        fth_destroy(c);
        return s2;
    };
#define FTH_CK_C(call, what)                                \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, what)); \
    } while (0)

    FTH_CK_C(cudaMemsetAsync(c->ws, 0, L.total, c->stream), "zero workspace");
    if (L.path != kPathDense64) {
        int lo = 0, hi = 0;
        FTH_CK_C(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
        FTH_CK_C(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, lo), "side stream");
        for (int b = 0; b < 2; ++b) {
            FTH_CK_C(cudaEventCreateWithFlags(&c->ev_filled[b], cudaEventDisableTiming), "event");
            FTH_CK_C(cudaEventCreateWithFlags(&c->ev_free[b], cudaEventDisableTiming), "event");
        }
        FTH_CK_C(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event");
    }

    // ---- M: dense matrices are validated and converted on the device (k_prepare.cu), from
    // the caller's device buffer directly or, for a host matrix, in chunks of rows staged
    // through the part of the workspace after M (zeroed again afterwards); sparse ones on
    // the host, where their structure is checked
    const int64_t N = L.N;
    const size_t esz_in = Min->dtype == FTH_F64 ? 8 : 4;
    if (Min->kind == FTH_DENSE) {
        const int layout = L.path == kPathDense64            ? kPrepF64
                           : L.precision == FTH_PREC_BF16X3  ? kPrepBf16x3
                           : L.precision == FTH_PREC_TF32    ? kPrepTf32
                                                             : kPrepF32;
        const int f64 = esz_in == 8 ? 1 : 0;
        if (Min->on_device) {
            FTH_CK_C(launch_dense_prepare(Min->values, f64, N, 0, N, L.Np, layout, c->M, c->Mlo, c->err,
                                          c->stream),
                     "prepare M");
        } else {
            uint8_t* stage = c->ws + L.off_q0;
            const size_t span = L.total - L.off_q0;
            const size_t row_bytes = (size_t)N * esz_in;
            if (span < row_bytes) {   // cannot happen: the state planes alone hold >= 16 N bytes
                c->last_error = "workspace too small to stage a row of M";
                return bail(FTH_E_WORKSPACE);
            }
            const int64_t rows = std::min<int64_t>(N, (int64_t)(span / row_bytes));
            for (int64_t r0 = 0; r0 < N; r0 += rows) {
                const int64_t nr = std::min<int64_t>(rows, N - r0);
                FTH_CK_C(cudaMemcpyAsync(stage, static_cast<const uint8_t*>(Min->values) + (size_t)r0 * row_bytes,
                                         (size_t)nr * row_bytes, cudaMemcpyHostToDevice, c->stream),
                         "h2d M");
                FTH_CK_C(launch_dense_prepare(stage, f64, N, r0, nr, L.Np, layout, c->M, c->Mlo, c->err,
                                              c->stream),
                         "prepare M");
            }
        }
        // the context's error word carries the flags here: no other kernel has run yet, and
        // the zeroing below clears it with the staging span
        uint32_t flags = 0;
        FTH_CK_C(cudaMemcpyAsync(&flags, c->err, 4, cudaMemcpyDeviceToHost, c->stream), "d2h flags");
        FTH_CK_C(cudaMemsetAsync(c->ws + L.off_q0, 0, L.total - L.off_q0, c->stream), "zero workspace");
        FTH_CK_C(cudaStreamSynchronize(c->stream), "sync");
        if (flags & kPrepNotSpd) {
            c->last_error = "M has a non-positive diagonal entry: not positive definite";
            return bail(FTH_E_NOT_SPD);
        }
        if (flags & kPrepNonFinite) {
            c->last_error = "M has non-finite entries";
            return bail(FTH_E_INVALID_ARG);
        }
    } else {
        const int64_t nnz = L.nnz;
        std::vector<int32_t> rp(N + 1), ci(std::max<int64_t>(nnz, 1));
        std::vector<uint8_t> raw((size_t)std::max<int64_t>(nnz, 1) * esz_in);
        if (Min->on_device) {
            FTH_CK_C(cudaMemcpy(rp.data(), Min->rowptr, (N + 1) * 4, cudaMemcpyDeviceToHost), "d2h rowptr");
            if (nnz) {
                FTH_CK_C(cudaMemcpy(ci.data(), Min->colind, nnz * 4, cudaMemcpyDeviceToHost), "d2h col");
                FTH_CK_C(cudaMemcpy(raw.data(), Min->values, nnz * esz_in, cudaMemcpyDeviceToHost), "d2h val");
            }
        } else {
            std::memcpy(rp.data(), Min->rowptr, (N + 1) * 4);
            if (nnz) {
                std::memcpy(ci.data(), Min->colind, nnz * 4);
                std::memcpy(raw.data(), Min->values, nnz * esz_in);
            }
        }
        if (rp[0] != 0 || rp[N] != nnz) {
            c->last_error = "CSR rowptr must start at 0 and end at nnz";
            return bail(FTH_E_INVALID_ARG);
        }
        std::vector<float> v(std::max<int64_t>(nnz, 1));
        for (int64_t i = 0; i < N; ++i) {
            if (rp[i + 1] < rp[i]) {
                c->last_error = "CSR rowptr not non-decreasing";
                return bail(FTH_E_INVALID_ARG);
            }
            bool diag = false;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                if (ci[e] < 0 || ci[e] >= N) {
                    c->last_error = "CSR column index out of range";
                    return bail(FTH_E_INVALID_ARG);
                }
                const double x = esz_in == 8 ? reinterpret_cast<const double*>(raw.data())[e]
                                             : (double)reinterpret_cast<const float*>(raw.data())[e];
                if (!std::isfinite(x)) {
                    c->last_error = "CSR values not finite";
                    return bail(FTH_E_INVALID_ARG);
                }
                v[e] = (float)x;
                if (ci[e] == i && x > 0.0) diag = true;
            }
            if (!diag) {
                c->last_error = "CSR row without a positive diagonal entry: not positive definite";
                return bail(FTH_E_NOT_SPD);
            }
        }
        FTH_CK_C(cudaMemcpyAsync(c->rowptr, rp.data(), (N + 1) * 4, cudaMemcpyHostToDevice, c->stream), "h2d rowptr");
        FTH_CK_C(cudaMemcpyAsync(c->col, ci.data(), std::max<int64_t>(nnz, 1) * 4, cudaMemcpyHostToDevice, c->stream), "h2d col");
        FTH_CK_C(cudaMemcpyAsync(c->val, v.data(), std::max<int64_t>(nnz, 1) * 4, cudaMemcpyHostToDevice, c->stream), "h2d val");
        FTH_CK_C(cudaStreamSynchronize(c->stream), "sync");
    }

    // ---- tracked pairs
    {
        std::vector<int32_t>& pr = c->reg_pairs;
        pr.reserve((size_t)L.ntracked * 2);
        auto add = [&](int64_t i, int64_t j) {
            if (i > j) std::swap(i, j);
            pr.push_back((int32_t)i);
            pr.push_back((int32_t)j);
        };
        if (L.track == FTH_TRACK_LIST) {
            for (int64_t e = 0; e < opt->npairs; ++e) add(opt->pairs[2 * e], opt->pairs[2 * e + 1]);
        } else if (L.track == FTH_TRACK_DIAG) {
            for (int64_t i = 0; i < N; ++i) add(i, i);
        } else if (L.path == kPathDense64) {
            for (int64_t i = 0; i < N; ++i)
                for (int64_t j = i; j < N; ++j) add(i, j);
        }
        if (!pr.empty()) {
            FTH_CK_C(cudaMemcpyAsync(c->pairs, pr.data(), pr.size() * 4, cudaMemcpyHostToDevice, c->stream), "h2d pairs");
            FTH_CK_C(cudaStreamSynchronize(c->stream), "sync");
        }
        if (c->prow) {
            // the same pairs grouped by their first index (counting sort over rows)
            const int64_t np = (int64_t)pr.size() / 2;
            std::vector<int32_t> prow((size_t)N + 1, 0), pcol((size_t)std::max<int64_t>(np, 1)),
                pe((size_t)std::max<int64_t>(np, 1));
            for (int64_t e = 0; e < np; ++e) ++prow[pr[2 * e] + 1];
            for (int64_t i = 0; i < N; ++i) prow[i + 1] += prow[i];
            std::vector<int32_t> fill(prow.begin(), prow.end() - 1);
            for (int64_t e = 0; e < np; ++e) {
                const int32_t k = fill[pr[2 * e]]++;
                pcol[k] = pr[2 * e + 1];
                pe[k] = (int32_t)e;
            }
            FTH_CK_C(cudaMemcpyAsync(c->prow, prow.data(), prow.size() * 4, cudaMemcpyHostToDevice, c->stream), "h2d prow");
            if (np) {
                FTH_CK_C(cudaMemcpyAsync(c->pcol, pcol.data(), np * 4, cudaMemcpyHostToDevice, c->stream), "h2d pcol");
                FTH_CK_C(cudaMemcpyAsync(c->pe, pe.data(), np * 4, cudaMemcpyHostToDevice, c->stream), "h2d pe");
            }
            FTH_CK_C(cudaStreamSynchronize(c->stream), "sync");
        }
    }

    // ---- tensor maps
    if (is_tc(c)) {
        const int kind = L.precision == FTH_PREC_TF32 ? 1 : 2;
        FTH_CK_C(tc_force_prepare(&c->tcf, kind, c->M, c->Mlo, c->ophi, c->oplo, L.Np, L.Rp, L.N, L.R,
                                  c->MQ),
                 "tensor maps (force)");
        if (L.track == FTH_TRACK_ALL) {
            float* tiles = static_cast<float*>(c->partial);
            FTH_CK_C(tc_syrk_prepare(&c->tcs, c->psb[0], L.Np, L.ps_ld, tiles), "tensor maps (syrk)");
            FTH_CK_C(tc_syrk_prepare(&c->tcs1, c->psb[1], L.Np, L.ps_ld, tiles), "tensor maps (syrk)");
        }
    }
#undef FTH_CK_C
    *out = c;
    return FTH_OK;
}

fth_status fth_run(fth_ctx* c, int64_t steps) {
    if (!c) return fail(nullptr, FTH_E_INVALID_ARG, "ctx is NULL");
    if (steps < 0) {
        c->last_error = "steps must be >= 0";
        return FTH_E_INVALID_ARG;
    }
    if (c->t + steps + 2 > (int64_t)0xFFFFFFFFll) {
        c->last_error = "kick index would exceed 2^32";
        return FTH_E_INVALID_ARG;
    }
    switch (c->L.path) {
        case kPathDense32: return run_dense32(c, steps);
        case kPathCsr: return run_csr(c, steps);
        default: return run_dense64(c, steps);
    }
}

fth_status fth_status_poll(fth_ctx* c) {
    if (!c) return fail(nullptr, FTH_E_INVALID_ARG, "ctx is NULL");
    uint32_t e = 0;
    FTH_CK(cudaMemcpyAsync(&e, c->err, 4, cudaMemcpyDeviceToHost, c->stream), "d2h err");
    FTH_CK(cudaStreamSynchronize(c->stream), "sync");
    if (e & kErrTimeout) {
        c->last_error = "a device wait timed out";
        return FTH_E_TIMEOUT;
    }
    if (e & kErrNonFinite) {
        c->last_error = "non-finite accumulator at a block flush";
        return FTH_E_NONFINITE;
    }
    return FTH_OK;
}

// Accumulator index of element (i, j), or a NOT_TRACKED / INVALID_ARG status.  `hint` is
// the position the caller expects (a request in registration order resolves without the
// map; the map is built on the first lookup that needs it).
static fth_status element_index(fth_ctx* c, int64_t i, int64_t j, int64_t* out,
                                int64_t hint = -1) {
    const Layout& L = c->L;
    if (i < 0 || j < 0 || i >= L.N || j >= L.N) {
        c->last_error = "pair index out of range";
        return FTH_E_INVALID_ARG;
    }
    if (L.track == FTH_TRACK_ALL && L.path == kPathDense32) {
        *out = packed_index(i, j, L.nbt);
        return FTH_OK;
    }
    const int64_t a = std::min(i, j), b = std::max(i, j);
    const std::vector<int32_t>& rp = c->reg_pairs;
    if (hint >= 0 && 2 * hint + 1 < (int64_t)rp.size() && rp[2 * hint] == a && rp[2 * hint + 1] == b) {
        *out = hint;
        return FTH_OK;
    }
    if (c->pair_index.empty() && !rp.empty()) {
        c->pair_index.reserve(rp.size() / 2);
        for (int64_t e = 0; 2 * e < (int64_t)rp.size(); ++e)
            c->pair_index.emplace(pair_key(rp[2 * e], rp[2 * e + 1]), e);
    }
    auto it = c->pair_index.find(pair_key(i, j));
    if (it == c->pair_index.end()) {
        c->last_error = "element (" + std::to_string(i) + ", " + std::to_string(j) + ") is not tracked";
        return FTH_E_NOT_TRACKED;
    }
    *out = it->second;
    return FTH_OK;
}

size_t fth_functional_bytes(int64_t nterms) {
    return nterms < 0 ? 0 : align256((size_t)nterms * 16 + 64);
}

fth_status fth_functional_add(fth_ctx* c, const int64_t* pairs, const double* weights,
                              int64_t nterms, void* device_buffer, size_t bytes, int64_t* id) {
    if (!c || !id || nterms < 0 || (nterms > 0 && (!pairs || !weights)) || !device_buffer)
        return fail(c ? &c->last_error : nullptr, FTH_E_INVALID_ARG, "bad functional arguments");
    if (bytes < fth_functional_bytes(nterms) || (reinterpret_cast<uintptr_t>(device_buffer) & 255u)) {
        c->last_error = "functional buffer too small or not 256-byte aligned";
        return FTH_E_WORKSPACE;
    }
    if (c->nblocks > 0 || c->inblock > 0) {
        c->last_error = "functionals must be added before the first sample is accumulated";
        return FTH_E_INVALID_ARG;
    }
    std::vector<int64_t> idx((size_t)nterms);
    for (int64_t k = 0; k < nterms; ++k) {
        const fth_status st = element_index(c, pairs[2 * k], pairs[2 * k + 1], &idx[k], k);
        if (st != FTH_OK) return st;
        if (!std::isfinite(weights[k])) {
            c->last_error = "non-finite functional weight";
            return FTH_E_INVALID_ARG;
        }
    }
    fth_ctx::Functional f;
    uint8_t* b = static_cast<uint8_t*>(device_buffer);
    f.acc = reinterpret_cast<double*>(b);
    f.idx = reinterpret_cast<int64_t*>(b + 64);
    f.w = reinterpret_cast<double*>(b + 64 + (size_t)nterms * 8);
    f.nterms = nterms;
    f.pairs.assign(pairs, pairs + 2 * nterms);
    f.weights.assign(weights, weights + nterms);
    FTH_CK(cudaMemsetAsync(f.acc, 0, 64, c->stream), "zero functional");
    if (nterms) {
        FTH_CK(cudaMemcpyAsync(f.idx, idx.data(), nterms * 8, cudaMemcpyHostToDevice, c->stream),
               "h2d functional idx");
        FTH_CK(cudaMemcpyAsync(f.w, weights, nterms * 8, cudaMemcpyHostToDevice, c->stream),
               "h2d functional weights");
    }
    FTH_CK(cudaStreamSynchronize(c->stream), "sync");
    c->funcs.push_back(std::move(f));
    *id = (int64_t)c->funcs.size() - 1;
    return FTH_OK;
}

// Terms of Tr O f(M) = <p^T O p> for a symmetric O of the context's order: w = O_ii on
// (i, i) and 2 O_ij on (i, j), i < j, from the entries on and above the diagonal (the
// lower triangle is the mirror and is not read); zero entries are dropped.  O NULL is the
// identity (Tr f(M)).  A device O is copied to the host first.
static fth_status operator_terms(fth_ctx* c, const fth_matrix* O, std::vector<int64_t>& pairs,
                                 std::vector<double>& w) {
    pairs.clear();
    w.clear();
    const int64_t n = c->L.N;
    if (!O) {
        for (int64_t i = 0; i < n; ++i) {
            pairs.push_back(i);
            pairs.push_back(i);
            w.push_back(1.0);
        }
        return FTH_OK;
    }
    if (O->n != n || (O->kind != FTH_DENSE && O->kind != FTH_CSR) ||
        (O->dtype != FTH_F32 && O->dtype != FTH_F64) || !O->values ||
        (O->kind == FTH_CSR && (!O->rowptr || !O->colind || O->nnz < 0))) {
        c->last_error = "operator: order, kind, dtype or pointers do not fit the context";
        return FTH_E_INVALID_ARG;
    }
    const size_t esz = O->dtype == FTH_F64 ? 8 : 4;
    const int64_t nv = O->kind == FTH_DENSE ? n * n : O->nnz;
    std::vector<uint8_t> vals((size_t)nv * esz);
    std::vector<int32_t> rp, ci;
    const int32_t* rowptr = O->rowptr;
    const int32_t* colind = O->colind;
    if (O->on_device) {
        FTH_CK(cudaMemcpy(vals.data(), O->values, vals.size(), cudaMemcpyDeviceToHost), "d2h O");
        if (O->kind == FTH_CSR) {
            rp.resize(n + 1);
            ci.resize(O->nnz);
            FTH_CK(cudaMemcpy(rp.data(), O->rowptr, rp.size() * 4, cudaMemcpyDeviceToHost), "d2h O");
            FTH_CK(cudaMemcpy(ci.data(), O->colind, ci.size() * 4, cudaMemcpyDeviceToHost), "d2h O");
            rowptr = rp.data();
            colind = ci.data();
        }
    } else if (nv > 0) {
        std::memcpy(vals.data(), O->values, vals.size());
    }
    auto value = [&](int64_t k) {
        return esz == 8 ? reinterpret_cast<const double*>(vals.data())[k]
                        : (double)reinterpret_cast<const float*>(vals.data())[k];
    };
    auto add = [&](int64_t i, int64_t j, double o) -> bool {
        if (!std::isfinite(o)) return false;
        if (o == 0.0) return true;
        pairs.push_back(i);
        pairs.push_back(j);
        w.push_back(i == j ? o : 2.0 * o);
        return true;
    };
    if (O->kind == FTH_DENSE) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i; j < n; ++j)
                if (!add(i, j, value(i * n + j))) {
                    c->last_error = "operator: non-finite entry";
                    return FTH_E_INVALID_ARG;
                }
    } else {
        if (rowptr[0] != 0 || rowptr[n] != O->nnz) {
            c->last_error = "operator: bad CSR row offsets";
            return FTH_E_INVALID_ARG;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (rowptr[i + 1] < rowptr[i]) {
                c->last_error = "operator: bad CSR row offsets";
                return FTH_E_INVALID_ARG;
            }
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                const int64_t j = colind[k];
                if (j < 0 || j >= n) {
                    c->last_error = "operator: CSR column out of range";
                    return FTH_E_INVALID_ARG;
                }
                if (j >= i && !add(i, j, value(k))) {
                    c->last_error = "operator: non-finite entry";
                    return FTH_E_INVALID_ARG;
                }
            }
        }
    }
    return FTH_OK;
}

fth_status fth_functional_operator_terms(fth_ctx* c, const fth_matrix* O, int64_t* nterms) {
    if (!c || !nterms) return fail(c ? &c->last_error : nullptr, FTH_E_INVALID_ARG, "NULL argument");
    std::vector<int64_t> pairs;
    std::vector<double> w;
    const fth_status st = operator_terms(c, O, pairs, w);
    if (st != FTH_OK) return st;
    *nterms = (int64_t)w.size();
    return FTH_OK;
}

fth_status fth_functional_add_operator(fth_ctx* c, const fth_matrix* O, void* device_buffer,
                                       size_t bytes, int64_t* id) {
    if (!c || !id) return fail(c ? &c->last_error : nullptr, FTH_E_INVALID_ARG, "NULL argument");
    std::vector<int64_t> pairs;
    std::vector<double> w;
    const fth_status st = operator_terms(c, O, pairs, w);
    if (st != FTH_OK) return st;
    return fth_functional_add(c, pairs.data(), w.data(), (int64_t)w.size(), device_buffer, bytes,
                              id);
}

fth_status fth_functional(fth_ctx* c, int64_t id, double* value, double* errbar) {
    if (!c || !value || id < 0 || id >= (int64_t)c->funcs.size())
        return fail(c ? &c->last_error : nullptr, FTH_E_INVALID_ARG, "bad functional id");
    const auto& f = c->funcs[id];
    std::vector<double> v((size_t)f.nterms);
    fth_status st = fth_elements(c, f.pairs.data(), f.nterms, v.data(), nullptr);
    if (st != FTH_OK) return st;
    double sum = 0.0;
    for (int64_t k = 0; k < f.nterms; ++k) sum += f.weights[k] * v[k];
    *value = f.nterms ? sum : 0.0;
    if (errbar) {
        double acc[3];
        FTH_CK(cudaMemcpyAsync(acc, f.acc, sizeof acc, cudaMemcpyDeviceToHost, c->stream),
               "d2h functional");
        FTH_CK(cudaStreamSynchronize(c->stream), "sync");
        const double nb = (double)c->nblocks;
        *errbar = nb >= 2 ? std::sqrt(acc[2] / (nb * (nb - 1.0))) : NAN;
    }
    return FTH_OK;
}

fth_status fth_elements(fth_ctx* c, const int64_t* pairs, int64_t k, double* values,
                        double* errbars) {
    if (!c) return fail(nullptr, FTH_E_INVALID_ARG, "ctx is NULL");
    if (k < 0 || (k > 0 && (!pairs || !values))) {
        c->last_error = "bad pairs / values";
        return FTH_E_INVALID_ARG;
    }
    fth_status st = fth_status_poll(c);
    if (st != FTH_OK) return st;
    const Layout& L = c->L;
    std::vector<int64_t> idx((size_t)k);
    for (int64_t e = 0; e < k; ++e) {
        st = element_index(c, pairs[2 * e], pairs[2 * e + 1], &idx[e], e);
        if (st != FTH_OK) return st;
    }
    const double nb = (double)c->nblocks;
    const double nacc = (double)(c->nblocks * c->block + c->inblock);
    std::vector<double> out((size_t)std::min(L.gcap, std::max<int64_t>(k, 1)) * 3);
    for (int64_t b0 = 0; b0 < k; b0 += L.gcap) {
        const int64_t m = std::min(L.gcap, k - b0);
        FTH_CK(cudaMemcpyAsync(c->gidx, idx.data() + b0, m * 8, cudaMemcpyHostToDevice, c->stream),
               "h2d idx");
        const bool p64 = L.path == kPathDense64;
        FTH_CK(launch_gather(c->gidx, m, c->mean, c->m2,
                             p64 ? nullptr : static_cast<const float*>(c->partial),
                             p64 ? static_cast<const double*>(c->partial) : nullptr, L.R, L.count,
                             c->gout, c->stream),
               "gather");
        FTH_CK(cudaMemcpyAsync(out.data(), c->gout, m * 3 * 8, cudaMemcpyDeviceToHost, c->stream),
               "d2h gather");
        FTH_CK(cudaStreamSynchronize(c->stream), "sync");
        for (int64_t e = 0; e < m; ++e) {
            const double mean = out[3 * e], m2 = out[3 * e + 1], part = out[3 * e + 2];
            const double total = mean * nb * (double)c->block * (double)L.R + part;
            values[b0 + e] = nacc > 0 ? total / (nacc * (double)L.R) : NAN;
            if (errbars) errbars[b0 + e] = nb >= 2 ? std::sqrt(m2 / (nb * (nb - 1.0))) : NAN;
        }
    }
    return FTH_OK;
}

fth_status fth_get_state(fth_ctx* c, int plane, double* host) {
    if (!c || !host) return fail(nullptr, FTH_E_INVALID_ARG, "NULL argument");
    const Layout& L = c->L;
    const int nsub = L.ns - 1;
    if (plane < FTH_PLANE_Q || plane > FTH_PLANE_S) {
        c->last_error = "bad plane";
        return FTH_E_INVALID_ARG;
    }
    const int nplanes = plane == FTH_PLANE_S ? nsub : 1;
    FTH_CK(cudaStreamSynchronize(c->stream), "sync");
    for (int a = 0; a < nplanes; ++a) {
        if (L.path == kPathDense64) {
            const double* src = static_cast<const double*>(
                plane == FTH_PLANE_Q ? c->q[0] : plane == FTH_PLANE_P ? c->p : c->s);
            src += (size_t)a * L.R * L.Np;
            std::vector<double> h((size_t)L.R * L.Np);
            FTH_CK(cudaMemcpy(h.data(), src, h.size() * 8, cudaMemcpyDeviceToHost), "d2h state");
            for (int64_t r = 0; r < L.R; ++r)
                for (int64_t i = 0; i < L.N; ++i)
                    host[((size_t)r * nplanes + a) * L.N + i] = h[r * L.Np + i];
        } else {
            const int64_t rows = L.path == kPathCsr ? L.N : L.Np;
            const float* src = static_cast<const float*>(
                plane == FTH_PLANE_Q ? c->q[c->cur] : plane == FTH_PLANE_P ? c->p : c->s);
            src += (size_t)a * rows * L.Rp;
            std::vector<float> h((size_t)L.N * L.Rp);
            FTH_CK(cudaMemcpy(h.data(), src, h.size() * 4, cudaMemcpyDeviceToHost), "d2h state");
            for (int64_t r = 0; r < L.R; ++r)
                for (int64_t i = 0; i < L.N; ++i)
                    host[((size_t)r * nplanes + a) * L.N + i] = h[i * L.Rp + r];
        }
    }
    return FTH_OK;
}

fth_status fth_set_state(fth_ctx* c, int plane, const double* host) {
    if (!c || !host) return fail(nullptr, FTH_E_INVALID_ARG, "NULL argument");
    const Layout& L = c->L;
    const int nsub = L.ns - 1;
    if (plane < FTH_PLANE_Q || plane > FTH_PLANE_S) {
        c->last_error = "bad plane";
        return FTH_E_INVALID_ARG;
    }
    const int nplanes = plane == FTH_PLANE_S ? nsub : 1;
    FTH_CK(cudaStreamSynchronize(c->stream), "sync");
    for (int a = 0; a < nplanes; ++a) {
        if (L.path == kPathDense64) {
            double* dst = static_cast<double*>(
                plane == FTH_PLANE_Q ? c->q[0] : plane == FTH_PLANE_P ? c->p : c->s);
            dst += (size_t)a * L.R * L.Np;
            std::vector<double> h((size_t)L.R * L.Np, 0.0);
            for (int64_t r = 0; r < L.R; ++r)
                for (int64_t i = 0; i < L.N; ++i) h[r * L.Np + i] = host[((size_t)r * nplanes + a) * L.N + i];
            FTH_CK(cudaMemcpy(dst, h.data(), h.size() * 8, cudaMemcpyHostToDevice), "h2d state");
        } else {
            const int64_t rows = L.path == kPathCsr ? L.N : L.Np;
            float* dst = static_cast<float*>(
                plane == FTH_PLANE_Q ? c->q[c->cur] : plane == FTH_PLANE_P ? c->p : c->s);
            dst += (size_t)a * rows * L.Rp;
            std::vector<float> h((size_t)L.N * L.Rp, 0.f);
            for (int64_t r = 0; r < L.R; ++r)
                for (int64_t i = 0; i < L.N; ++i) h[i * L.Rp + r] = (float)host[((size_t)r * nplanes + a) * L.N + i];
            FTH_CK(cudaMemcpy(dst, h.data(), h.size() * 4, cudaMemcpyHostToDevice), "h2d state");
        }
    }
    if (plane == FTH_PLANE_Q) return upload_state_operand(c);
    return FTH_OK;
}

fth_status fth_info(const fth_ctx* c, fth_info_t* info) {
    if (!c || !info) return fail(nullptr, FTH_E_INVALID_ARG, "NULL argument");
    info->steps = c->t;
    info->samples = c->nsamp;
    info->accumulated = c->accumulated;
    info->blocks = c->nblocks;
    info->launches = c->launches;
    info->primed = c->primed;
    info->precision = c->L.precision;
    info->n = c->L.N;
    info->replicas = c->L.R;
    info->tracked = c->L.count;
    info->workspace_bytes = c->L.total;
    return FTH_OK;
}

fth_status fth_test_stall(fth_ctx* c, uint64_t limit_ns) {
    if (!c) return fail(nullptr, FTH_E_INVALID_ARG, "ctx is NULL");
    if (!is_tc(c) || !c->tcf) {
        c->last_error = "fth_test_stall needs a tensor-core (TF32 or BF16X3) dense context";
        return FTH_E_UNSUPPORTED;
    }
    if (limit_ns > 1000000000ull) {
        c->last_error = "stall limit above the 1 s wait bound";
        return FTH_E_INVALID_ARG;
    }
    tc_force_set_stall(c->tcf, limit_ns);
    return FTH_OK;
}

fth_status fth_profile_enable(fth_ctx* c, int enable) {
    if (!c) return fail(nullptr, FTH_E_INVALID_ARG, "ctx is NULL");
    c->prof = enable != 0;
    return FTH_OK;
}

fth_status fth_profile_read(fth_ctx* c, double* ms, int64_t* launches) {
    if (!c || !ms || !launches) return fail(nullptr, FTH_E_INVALID_ARG, "NULL argument");
    FTH_CK(cudaStreamSynchronize(c->stream), "sync");
    for (auto& r : c->prof_recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            c->prof_ms[r.cls] += t;
            c->prof_n[r.cls] += 1;
        }
        c->prof_pool.push_back(r.a);
        c->prof_pool.push_back(r.b);
    }
    c->prof_recs.clear();
    for (int k = 0; k < FTH_K_CLASSES; ++k) {
        ms[k] = c->prof_ms[k];
        launches[k] = c->prof_n[k];
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    return FTH_OK;
}

void fth_destroy(fth_ctx* c) {
    if (!c) return;
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    for (int b = 0; b < 2; ++b) {
        if (c->ev_filled[b]) cudaEventDestroy(c->ev_filled[b]);
        if (c->ev_free[b]) cudaEventDestroy(c->ev_free[b]);
    }
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->tcs1) tc_syrk_free(c->tcs1);
    for (auto& r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->prof_pool) cudaEventDestroy(e);
    if (c->tcf) tc_force_free(c->tcf);
    if (c->tcs) tc_syrk_free(c->tcs);
    delete c;
}

}  // extern "C"
