// Problem pools, host side: admission into a slab of the caller's workspace, device
// descriptor table, work lists, the per-step launch sequence (replayed from captured
// CUDA graphs), an autotuner for the force kernel, and per-problem results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "fth.h"
#include "fth_internal.h"
#include "pool_internal.h"

using namespace fth;

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
int64_t rup(int64_t x, int64_t m) { return ((x + m - 1) / m) * m; }

struct Layout {
    size_t a_hi = 0, a_lo = 0, bt_hi = 0, bt_lo = 0, mq = 0, q0 = 0, q1 = 0, p = 0, s = 0, x = 0;
    size_t rowptr = 0, col = 0, val = 0, pairs = 0, partial = 0, mean = 0, m2 = 0, total = 0;
};

Layout problem_layout(int kind, int64_t n, int64_t nnz, int ns, int64_t R, int prec,
                      int64_t npairs) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o = a256(o + std::max<size_t>(b, 1));
        return at;
    };
    const size_t plane = (size_t)n * R * 4;
    if (kind == FTH_DENSE) {
        const int64_t np = rup(n, 128), nb = np / 128;
        const size_t esz = prec == FTH_PREC_TF32 ? 4 : 2;
        // BF16X3 stores the upper 128 x 128 blocks only (32 KiB each per plane)
        const size_t mbytes = prec == FTH_PREC_BF16X3 ? (size_t)(nb * (nb + 1) / 2) * 32768
                                                      : (size_t)np * np * esz;
        L.a_hi = take(mbytes);
        if (prec == FTH_PREC_BF16X3) L.a_lo = take(mbytes);
        L.bt_hi = take((size_t)np * R * esz);
        if (prec == FTH_PREC_BF16X3) L.bt_lo = take((size_t)np * R * esz);
        L.mq = take(plane);
        L.q0 = take(plane);
    } else {
        L.rowptr = take((size_t)(n + 1) * 4);
        L.col = take((size_t)nnz * 4);
        L.val = take((size_t)nnz * 4);
        L.q0 = take(plane);
        L.q1 = take(plane);
    }
    L.p = take(plane);
    L.s = take(plane * std::max(ns - 1, 1));
    L.x = take(plane);
    L.pairs = take((size_t)npairs * 8);
    L.partial = take((size_t)npairs * 4);
    L.mean = take((size_t)npairs * 8);
    L.m2 = take((size_t)npairs * 8);
    L.total = o;
    return L;
}

struct Problem {
    bool used = false;
    PoolDesc h{};            // host mirror (constants and pointers; counters live on device)
    size_t off = 0, bytes = 0;
    int64_t npairs = 0;
    std::unordered_map<uint64_t, int64_t> pair_index;
};

uint64_t pkey(int64_t i, int64_t j) {
    if (i > j) std::swap(i, j);
    return ((uint64_t)i << 32) | (uint64_t)j;
}

}  // namespace

struct fth_pool {
    int64_t R = 32;
    int prec = FTH_PREC_BF16X3;
    int kind_tc = 2;
    int64_t max_problems = 0, graph_steps = 0;
    cudaStream_t stream = nullptr;
    uint8_t* ws = nullptr;
    size_t ws_bytes = 0;
    PoolDesc* d_desc = nullptr;
    PoolForceItem* d_force = nullptr;
    PoolRowItem* d_rows = nullptr;     // dense rows, then CSR rows
    PoolAccItem* d_acc = nullptr;
    int* d_live = nullptr;                // live slots (progress kernel)
    double* d_prog = nullptr;             // [max_problems][2] progress output
    uint8_t* stage = nullptr;             // kPoolStageBytes for dense uploads
    uint32_t* d_err = nullptr;
    int64_t cap_force = 0, cap_rows = 0, cap_acc = 0;
    size_t slab_begin = 0, slab_end = 0;
    std::map<size_t, size_t> free_list;   // offset -> bytes
    size_t used_bytes = 0;
    std::vector<Problem> probs;
    std::vector<PoolForceItem> h_force;
    std::vector<PoolRowItem> h_rows;
    std::vector<PoolAccItem> h_acc;
    std::vector<int> h_live;
    int64_t n_force = 0, n_dense_rows = 0, n_csr_rows = 0;
    // row items grouped by shared GLE constants: one GLE (and one CSR) launch per group
    struct Group {
        GleF32 g;
        int ns;
        int64_t dense_begin, dense_count, csr_begin, csr_count;
    };
    std::vector<Group> groups;
    bool dirty = true;
    bool tuned = false;
    int variant = 0, grid = 152;
    int64_t tuned_items = 0;   // force-list length the tuning was done on
    double tuned_us = 0.0;
    int gle_variant = 1;
    bool gle_tuned = false;
    double gle_us = 0.0;
    int sms = 152;
    cudaGraphExec_t gexec = nullptr;
    bool graph_valid = false;
    int64_t graphs = 0;
    std::string last_error;
};

namespace {

fth_status perr(fth_pool* P, fth_status st, const std::string& m) {
    if (P) P->last_error = m;
    return st;
}

#define PCK(call, what)                                                                 \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return perr(P, FTH_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool slab_alloc(fth_pool* P, size_t bytes, size_t* off) {
    for (auto it = P->free_list.begin(); it != P->free_list.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t roff = it->first + bytes;
            P->free_list.erase(it);
            if (rest > 0) P->free_list[roff] = rest;
            P->used_bytes += bytes;
            return true;
        }
    }
    return false;
}

void slab_free(fth_pool* P, size_t off, size_t bytes) {
    P->used_bytes -= bytes;
    auto it = P->free_list.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != P->free_list.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        P->free_list.erase(nx);
    }
    if (it != P->free_list.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            P->free_list.erase(it);
        }
    }
}

fth_status check_problem(const fth_pool* P, const fth_matrix* M, const fth_gle* gle,
                         const fth_problem_options* po) {
    if (!M || !gle || !po || !M->values) return FTH_E_INVALID_ARG;
    if (M->n < 1 || M->n > (1 << 24)) return FTH_E_INVALID_ARG;
    if (M->kind != FTH_DENSE && M->kind != FTH_CSR) return FTH_E_INVALID_ARG;
    if (M->dtype != FTH_F32 && M->dtype != FTH_F64) return FTH_E_INVALID_ARG;
    if (M->kind == FTH_CSR && (!M->rowptr || !M->colind || M->nnz < 0)) return FTH_E_INVALID_ARG;
    if (gle->s < 0 || gle->s > 4) return FTH_E_UNSUPPORTED;
    if (!(po->dt > 0.0) || po->block < 1 || po->burnin < 0 || po->npairs < 0) return FTH_E_INVALID_ARG;
    if (po->npairs > 0 && !po->pairs) return FTH_E_INVALID_ARG;
    if (po->observable != FTH_OBS_P && po->observable != FTH_OBS_Q) return FTH_E_INVALID_ARG;
    if (po->replica_offset < 0 || po->replica_offset + P->R > (1ll << 32)) return FTH_E_INVALID_ARG;
    for (int64_t e = 0; e < po->npairs; ++e) {
        const int64_t i = po->pairs[2 * e], j = po->pairs[2 * e + 1];
        if (i < 0 || j < 0 || i >= M->n || j >= M->n) return FTH_E_INVALID_ARG;
    }
    return FTH_OK;
}

fth_status rebuild_lists(fth_pool* P) {
    P->h_force.clear();
    P->h_rows.clear();
    P->h_live.clear();
    P->h_acc.clear();
    P->groups.clear();
    // the GLE constants of a problem up to (not including) its noise keys
    const size_t key_bytes = offsetof(GleF32, key0);
    auto group_of = [&](const PoolDesc& d) {
        for (size_t k = 0; k < P->groups.size(); ++k)
            if (P->groups[k].ns == d.ns && std::memcmp(&P->groups[k].g, &d.g, key_bytes) == 0)
                return (int)k;
        fth_pool::Group gr{};
        gr.g = d.g;
        gr.ns = d.ns;
        P->groups.push_back(gr);
        return (int)P->groups.size() - 1;
    };
    std::vector<std::vector<PoolRowItem>> dense_by(0), csr_by(0);
    for (int b = 0; b < (int)P->probs.size(); ++b) {
        const Problem& pr = P->probs[b];
        if (!pr.used) continue;
        P->h_live.push_back(b);
        const int n = pr.h.n;
        const int np = (int)pr.npairs;
        const int nch = std::max(1, (np + kPoolAccChunk - 1) / kPoolAccChunk);
        for (int c = 0; c < nch; ++c)
            P->h_acc.push_back({b, c * kPoolAccChunk, std::min(np, (c + 1) * kPoolAccChunk), nch});
        const int gi = group_of(pr.h);
        dense_by.resize(P->groups.size());
        csr_by.resize(P->groups.size());
        if (pr.h.kind == 0) {
            for (int rb = 0; rb < (n + 127) / 128; ++rb) P->h_force.push_back({b, rb});
            for (int r0 = 0; r0 < n; r0 += 32) dense_by[gi].push_back({b, r0});
        } else {
            for (int r0 = 0; r0 < n; r0 += 32) csr_by[gi].push_back({b, r0});
        }
    }
    for (size_t k = 0; k < P->groups.size(); ++k) {
        P->groups[k].dense_begin = (int64_t)P->h_rows.size();
        P->groups[k].dense_count = (int64_t)dense_by[k].size();
        P->h_rows.insert(P->h_rows.end(), dense_by[k].begin(), dense_by[k].end());
    }
    const int64_t n_dense = (int64_t)P->h_rows.size();
    for (size_t k = 0; k < P->groups.size(); ++k) {
        P->groups[k].csr_begin = (int64_t)P->h_rows.size();
        P->groups[k].csr_count = (int64_t)csr_by[k].size();
        P->h_rows.insert(P->h_rows.end(), csr_by[k].begin(), csr_by[k].end());
    }
    // longest K first, then round-robin over the persistent CTAs (LPT-like balance)
    std::stable_sort(P->h_force.begin(), P->h_force.end(),
                     [&](const PoolForceItem& a, const PoolForceItem& b) {
                         return P->probs[a.problem].h.np > P->probs[b.problem].h.np;
                     });
    P->n_force = (int64_t)P->h_force.size();
    P->n_dense_rows = n_dense;
    P->n_csr_rows = (int64_t)P->h_rows.size() - n_dense;
    if (P->n_force > P->cap_force || (int64_t)P->h_rows.size() > P->cap_rows ||
        (int64_t)P->h_acc.size() > P->cap_acc)
        return perr(P, FTH_E_WORKSPACE, "work lists exceed the pool's capacity");
    if (!P->h_force.empty())
        PCK(cudaMemcpyAsync(P->d_force, P->h_force.data(), P->h_force.size() * sizeof(PoolForceItem),
                            cudaMemcpyHostToDevice, P->stream), "h2d force items");
    if (!P->h_rows.empty())
        PCK(cudaMemcpyAsync(P->d_rows, P->h_rows.data(), P->h_rows.size() * sizeof(PoolRowItem),
                            cudaMemcpyHostToDevice, P->stream), "h2d row items");
    if (!P->h_live.empty())
        PCK(cudaMemcpyAsync(P->d_live, P->h_live.data(), P->h_live.size() * sizeof(int),
                            cudaMemcpyHostToDevice, P->stream), "h2d live slots");
    if (!P->h_acc.empty())
        PCK(cudaMemcpyAsync(P->d_acc, P->h_acc.data(), P->h_acc.size() * sizeof(PoolAccItem),
                            cudaMemcpyHostToDevice, P->stream), "h2d accumulate items");
    PCK(cudaStreamSynchronize(P->stream), "sync");
    P->dirty = false;
    P->graph_valid = false;
    return FTH_OK;
}

// One pool step.  With `ev` set, an event pair brackets each launch: ev[2c], ev[2c+1]
// for kernel class c (fth_pool_kernel).
fth_status enqueue_step(fth_pool* P, cudaEvent_t* ev = nullptr) {
    auto mark = [&](int c, int end) {
        return ev ? cudaEventRecord(ev[2 * c + end], P->stream) : cudaSuccess;
    };
    if (P->n_force > 0) {
        PCK(mark(FTH_PK_FORCE, 0), "event");
        PCK(launch_pool_force(P->kind_tc, (int)P->R, P->variant, P->d_desc, P->d_force,
                              (int)P->n_force, P->grid, P->d_err, P->stream), "pool force");
        PCK(mark(FTH_PK_FORCE, 1), "event");
    }
    if (P->n_dense_rows > 0) {
        PCK(mark(FTH_PK_GLE, 0), "event");
        for (const auto& gr : P->groups)
            if (gr.dense_count > 0)
                PCK(launch_pool_gle(P->gle_variant, P->d_desc, P->d_rows + gr.dense_begin,
                                    (int)gr.dense_count, (int)P->R, P->kind_tc, gr.ns, gr.g,
                                    P->stream), "pool gle");
        PCK(mark(FTH_PK_GLE, 1), "event");
    }
    if (P->n_csr_rows > 0) {
        PCK(mark(FTH_PK_CSR, 0), "event");
        for (const auto& gr : P->groups)
            if (gr.csr_count > 0)
                PCK(launch_pool_csr(P->d_desc, P->d_rows + gr.csr_begin, (int)gr.csr_count,
                                    (int)P->R, gr.ns, gr.g, P->stream), "pool csr");
        PCK(mark(FTH_PK_CSR, 1), "event");
    }
    PCK(mark(FTH_PK_ACCUM, 0), "event");
    PCK(launch_pool_accum(P->d_desc, P->d_acc, (int)P->h_acc.size(), (int)P->R, P->d_err,
                          P->stream), "pool accumulate");
    PCK(mark(FTH_PK_ACCUM, 1), "event");
    return FTH_OK;
}

// Autotuner: time each force-kernel configuration (pipeline depth with one or two
// CTAs per SM, persistent grid of 1 or 2 waves) on the pool's current work list and keep
// the fastest.  The force kernel only reads state and rewrites M q, so the extra launches
// change no result.
fth_status autotune(fth_pool* P) {
    if (P->n_force == 0) return FTH_OK;
    struct Cand {
        int variant, grid;
    };
    std::vector<Cand> cands = {{0, P->sms}, {1, P->sms}, {1, 2 * P->sms}};
    cudaEvent_t e0, e1;
    PCK(cudaEventCreate(&e0), "event");
    PCK(cudaEventCreate(&e1), "event");
    double best = 1e30;
    for (const Cand& c : cands) {
        const int g = (int)std::min<int64_t>(c.grid, P->n_force);
        PCK(launch_pool_force(P->kind_tc, (int)P->R, c.variant, P->d_desc, P->d_force,
                              (int)P->n_force, g, P->d_err, P->stream), "autotune");
        PCK(cudaEventRecord(e0, P->stream), "event");
        for (int k = 0; k < 3; ++k)
            PCK(launch_pool_force(P->kind_tc, (int)P->R, c.variant, P->d_desc, P->d_force,
                                  (int)P->n_force, g, P->d_err, P->stream), "autotune");
        PCK(cudaEventRecord(e1, P->stream), "event");
        PCK(cudaEventSynchronize(e1), "event");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double us = ms * 1e3 / 3.0;
        if (us < best) {
            best = us;
            P->variant = c.variant;
            P->grid = g;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P->tuned_us = best;
    P->tuned_items = P->n_force;
    P->tuned = true;
    P->graph_valid = false;
    return FTH_OK;
}

// The dense GLE kernel's variants differ only in how lanes map onto elements, so they
// give identical results: time each on real steps (kGleReps steps apiece, the fastest
// launch counts) and keep the fastest.  These steps are part of the run that asked.
constexpr int kGleReps = 3;
constexpr int64_t kGleTuneSteps = (int64_t)kPoolGleVariants * kGleReps;

fth_status autotune_gle(fth_pool* P) {
    cudaEvent_t ev[2 * FTH_PK_CLASSES];
    for (auto& e : ev) PCK(cudaEventCreate(&e), "event");
    double best = 1e30;
    int pick = P->gle_variant;
    fth_status st = FTH_OK;
    for (int v = 0; v < kPoolGleVariants && st == FTH_OK; ++v) {
        P->gle_variant = v;
        double vbest = 1e30;
        for (int k = 0; k < kGleReps && st == FTH_OK; ++k) {
            st = enqueue_step(P, ev);
            if (st == FTH_OK && cudaStreamSynchronize(P->stream) != cudaSuccess)
                st = perr(P, FTH_E_CUDA, "sync");
            float ms = 0.f;
            if (st == FTH_OK) cudaEventElapsedTime(&ms, ev[2 * FTH_PK_GLE], ev[2 * FTH_PK_GLE + 1]);
            vbest = std::min(vbest, (double)ms * 1e3);
        }
        if (vbest < best) {
            best = vbest;
            pick = v;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    P->gle_variant = pick;
    P->gle_us = best;
    P->gle_tuned = true;
    P->graph_valid = false;
    return st;
}

}  // namespace

extern "C" {

fth_status fth_pool_create(const fth_pool_options* opt, void* workspace, size_t bytes,
                           fth_pool** out) {
    if (!opt || !out) return FTH_E_INVALID_ARG;
    *out = nullptr;
    if (opt->replicas != 32 && opt->replicas != 64 && opt->replicas != 128) return FTH_E_UNSUPPORTED;
    if (opt->precision != FTH_PREC_BF16X3 && opt->precision != FTH_PREC_TF32) return FTH_E_UNSUPPORTED;
    if (opt->max_problems < 1 || opt->graph_steps < 0) return FTH_E_INVALID_ARG;
    if (opt->graph_steps > 0 && !opt->stream) return FTH_E_INVALID_ARG;   // no capture on stream 0
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return FTH_E_WORKSPACE;
    fth_pool* P = new fth_pool();
    P->R = opt->replicas;
    P->prec = opt->precision;
    P->kind_tc = opt->precision == FTH_PREC_TF32 ? 1 : 2;
    P->max_problems = opt->max_problems;
    P->graph_steps = opt->graph_steps;
    P->stream = static_cast<cudaStream_t>(opt->stream);
    P->ws = static_cast<uint8_t*>(workspace);
    P->ws_bytes = bytes;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, dev);
    // header: descriptors, work lists (sized from the workspace: every 128-row block of a
    // dense problem needs >= 64 KiB of M, every 32 rows >= 32 R 4 B of state), error word
    const size_t min_problem = a256((size_t)32 * P->R * 4);
    P->cap_force = (int64_t)(bytes / 65536) + P->max_problems;
    P->cap_rows = (int64_t)(bytes / (min_problem * 4)) + P->max_problems;
    // a tracked pair takes >= 28 bytes of a problem's slab (indices, partial, mean, M2)
    P->cap_acc = (int64_t)(bytes / (28 * (size_t)kPoolAccChunk)) + P->max_problems;
    size_t o = 0;
    const size_t off_desc = o;
    o = a256(o + sizeof(PoolDesc) * (size_t)P->max_problems);
    const size_t off_force = o;
    o = a256(o + sizeof(PoolForceItem) * (size_t)P->cap_force);
    const size_t off_rows = o;
    o = a256(o + sizeof(PoolRowItem) * (size_t)P->cap_rows);
    const size_t off_acc = o;
    o = a256(o + sizeof(PoolAccItem) * (size_t)P->cap_acc);
    const size_t off_live = o;
    o = a256(o + sizeof(int) * (size_t)P->max_problems);
    const size_t off_prog = o;
    o = a256(o + 2 * sizeof(double) * (size_t)P->max_problems);
    const size_t off_stage = o;
    o = a256(o + kPoolStageBytes);
    const size_t off_err = o;
    o = a256(o + 256);
    if (o >= bytes) {
        delete P;
        return FTH_E_WORKSPACE;
    }
    P->d_desc = reinterpret_cast<PoolDesc*>(P->ws + off_desc);
    P->d_force = reinterpret_cast<PoolForceItem*>(P->ws + off_force);
    P->d_rows = reinterpret_cast<PoolRowItem*>(P->ws + off_rows);
    P->d_acc = reinterpret_cast<PoolAccItem*>(P->ws + off_acc);
    P->d_err = reinterpret_cast<uint32_t*>(P->ws + off_err);
    P->stage = P->ws + off_stage;
    P->d_live = reinterpret_cast<int*>(P->ws + off_live);
    P->d_prog = reinterpret_cast<double*>(P->ws + off_prog);
    P->slab_begin = o;
    P->slab_end = bytes & ~size_t(255);
    P->free_list[P->slab_begin] = P->slab_end - P->slab_begin;
    P->probs.resize((size_t)P->max_problems);
    if (cudaMemsetAsync(P->ws, 0, o, P->stream) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) {
        delete P;
        return FTH_E_CUDA;
    }
    *out = P;
    return FTH_OK;
}

fth_status fth_pool_footprint(const fth_pool* P, const fth_matrix* M, const fth_gle* gle,
                              const fth_problem_options* po, size_t* bytes) {
    if (!P || !bytes) return FTH_E_INVALID_ARG;
    const fth_status st = check_problem(P, M, gle, po);
    if (st != FTH_OK) return st;
    *bytes = problem_layout(M->kind, M->n, M->nnz, gle->s + 1, P->R, P->prec, po->npairs).total;
    return FTH_OK;
}

fth_status fth_pool_add(fth_pool* P, const fth_matrix* M, const fth_gle* gle,
                        const fth_problem_options* po, int64_t* handle) {
    if (!P || !handle) return FTH_E_INVALID_ARG;
    fth_status st = check_problem(P, M, gle, po);
    if (st != FTH_OK) return perr(P, st, "invalid problem");
    int slot = -1;
    for (int b = 0; b < (int)P->probs.size(); ++b)
        if (!P->probs[b].used) {
            slot = b;
            break;
        }
    if (slot < 0) return perr(P, FTH_E_WORKSPACE, "problem table full");
    const int ns = gle->s + 1;
    const int64_t n = M->n, R = P->R;
    const Layout L = problem_layout(M->kind, n, M->nnz, ns, R, P->prec, po->npairs);
    size_t off = 0;
    if (!slab_alloc(P, L.total, &off))
        return perr(P, FTH_E_WORKSPACE, "not admitted: footprint exceeds the free workspace");
    uint8_t* base = P->ws + off;
    // the slab range may have belonged to a problem whose last launches are still queued
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) {
        slab_free(P, off, L.total);
        return perr(P, FTH_E_CUDA, "sync");
    }
    auto fail_free = [&](fth_status s2, const std::string& m) {
        slab_free(P, off, L.total);
        return perr(P, s2, m);
    };
    // O half-step constants (FP64, library propagator)
    double T[25], S[25];
    st = fth_gle_propagator(gle, po->dt, T, S);
    if (st != FTH_OK) return fail_free(st, "invalid GLE");
    Problem pr;
    pr.used = true;
    pr.off = off;
    pr.bytes = L.total;
    pr.npairs = po->npairs;
    PoolDesc& d = pr.h;
    std::memset(&d, 0, sizeof d);
    fill_gle_constants(ns, T, S, &d.g, nullptr);
    d.g.dt = (float)po->dt;
    d.g.hdt = (float)(0.5 * po->dt);
    d.g.key0 = (uint32_t)po->seed;
    d.g.key1 = (uint32_t)(po->seed >> 32);
    d.g.roff = (uint32_t)po->replica_offset;
    set_round_keys(d.g);
    d.kind = M->kind == FTH_DENSE ? 0 : 1;
    d.n = (int)n;
    d.np = (int)(M->kind == FTH_DENSE ? rup(n, 128) : n);
    d.ns = ns;
    d.observable = po->observable;
    d.npairs = (int)po->npairs;
    d.live = 1;
    d.sym = (M->kind == FTH_DENSE && P->prec == FTH_PREC_BF16X3) ? 1 : 0;
    d.burnin = po->burnin;
    d.block = po->block;
    d.mq = L.mq ? reinterpret_cast<float*>(base + L.mq) : nullptr;
    d.q[0] = reinterpret_cast<float*>(base + L.q0);
    d.q[1] = L.q1 ? reinterpret_cast<float*>(base + L.q1) : d.q[0];
    d.p = reinterpret_cast<float*>(base + L.p);
    d.s = reinterpret_cast<float*>(base + L.s);
    d.x = reinterpret_cast<float*>(base + L.x);
    d.pairs = reinterpret_cast<int32_t*>(base + L.pairs);
    d.partial = reinterpret_cast<float*>(base + L.partial);
    d.mean = reinterpret_cast<double*>(base + L.mean);
    d.m2 = reinterpret_cast<double*>(base + L.m2);
    // zero before the uploads below, which use synchronous copies (another stream)
    if (cudaMemsetAsync(base, 0, L.total, P->stream) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess)
        return fail_free(FTH_E_CUDA, "zero problem memory");

    // dense M: checked on the host (diagonal), converted on the device row block by row
    // block (FP32 / FP64 rows staged through the pool's staging buffer when on the host)
    const size_t esz_in = M->dtype == FTH_F64 ? 8 : 4;
    auto value_at = [&](const std::vector<uint8_t>& raw, size_t k) {
        return esz_in == 8 ? reinterpret_cast<const double*>(raw.data())[k]
                           : (double)reinterpret_cast<const float*>(raw.data())[k];
    };
    if (M->kind == FTH_DENSE) {
        std::vector<uint8_t> diag((size_t)n * esz_in);
        if (M->on_device) {
            if (cudaMemcpy2D(diag.data(), esz_in, M->values, (size_t)(n + 1) * esz_in, esz_in, (size_t)n,
                             cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail_free(FTH_E_CUDA, "d2h diagonal");
        } else {
            for (int64_t i = 0; i < n; ++i)
                std::memcpy(diag.data() + i * esz_in,
                            static_cast<const uint8_t*>(M->values) + (size_t)(i * n + i) * esz_in, esz_in);
        }
        for (int64_t i = 0; i < n; ++i)
            if (!(value_at(diag, (size_t)i) > 0.0))
                return fail_free(FTH_E_NOT_SPD, "M has a non-positive diagonal entry");
        d.a_hi = base + L.a_hi;
        d.bt_hi = base + L.bt_hi;
        if (P->prec == FTH_PREC_BF16X3) {
            d.a_lo = base + L.a_lo;
            d.bt_lo = base + L.bt_lo;
        }
        const int rows_per = (int)std::max<int64_t>(1, (int64_t)(kPoolStageBytes / ((size_t)n * esz_in)));
        for (int64_t r0 = 0; r0 < n; r0 += rows_per) {
            const int nr = (int)std::min<int64_t>(rows_per, n - r0);
            const uint8_t* src = static_cast<const uint8_t*>(M->values) + (size_t)r0 * n * esz_in;
            const void* dsrc = src;
            if (!M->on_device) {
                if (cudaMemcpyAsync(P->stage, src, (size_t)nr * n * esz_in, cudaMemcpyHostToDevice,
                                    P->stream) != cudaSuccess)
                    return fail_free(FTH_E_CUDA, "h2d M rows");
                dsrc = P->stage;
            }
            if (launch_pool_convert(dsrc, esz_in == 8, (int)n, d.np, (int)r0, nr, P->kind_tc,
                                    d.a_hi, d.a_lo, P->stream) != cudaSuccess)
                return fail_free(FTH_E_CUDA, "convert M");
        }
    } else {
        const int64_t nnz = M->nnz;
        std::vector<int32_t> rp(n + 1), ci((size_t)std::max<int64_t>(nnz, 1));
        std::vector<uint8_t> raw((size_t)std::max<int64_t>(nnz, 1) * esz_in);
        if (M->on_device) {
            if (cudaMemcpy(rp.data(), M->rowptr, (n + 1) * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                (nnz && cudaMemcpy(ci.data(), M->colind, nnz * 4, cudaMemcpyDeviceToHost) != cudaSuccess) ||
                (nnz && cudaMemcpy(raw.data(), M->values, nnz * esz_in, cudaMemcpyDeviceToHost) != cudaSuccess))
                return fail_free(FTH_E_CUDA, "d2h CSR");
        } else {
            std::memcpy(rp.data(), M->rowptr, (n + 1) * 4);
            if (nnz) {
                std::memcpy(ci.data(), M->colind, nnz * 4);
                std::memcpy(raw.data(), M->values, nnz * esz_in);
            }
        }
        if (rp[0] != 0 || rp[n] != nnz) return fail_free(FTH_E_INVALID_ARG, "CSR rowptr");
        std::vector<float> v((size_t)std::max<int64_t>(nnz, 1));
        for (int64_t i = 0; i < n; ++i) {
            if (rp[i + 1] < rp[i]) return fail_free(FTH_E_INVALID_ARG, "CSR rowptr order");
            bool diag = false;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                if (ci[e] < 0 || ci[e] >= n) return fail_free(FTH_E_INVALID_ARG, "CSR column");
                const double x = value_at(raw, (size_t)e);
                v[e] = (float)x;
                if (ci[e] == i && x > 0.0) diag = true;
            }
            if (!diag) return fail_free(FTH_E_NOT_SPD, "CSR row without a positive diagonal");
        }
        d.rowptr = reinterpret_cast<int32_t*>(base + L.rowptr);
        d.col = reinterpret_cast<int32_t*>(base + L.col);
        d.val = reinterpret_cast<float*>(base + L.val);
        if (cudaMemcpy(const_cast<int32_t*>(d.rowptr), rp.data(), (n + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            (nnz && cudaMemcpy(const_cast<int32_t*>(d.col), ci.data(), nnz * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
            (nnz && cudaMemcpy(const_cast<float*>(d.val), v.data(), nnz * 4, cudaMemcpyHostToDevice) != cudaSuccess))
            return fail_free(FTH_E_CUDA, "h2d CSR");
    }
    // tracked pairs
    std::vector<int32_t> pp((size_t)po->npairs * 2);
    for (int64_t e = 0; e < po->npairs; ++e) {
        int64_t i = po->pairs[2 * e], j = po->pairs[2 * e + 1];
        if (i > j) std::swap(i, j);
        pr.pair_index.emplace(pkey(i, j), e);
        pp[2 * e] = (int32_t)i;
        pp[2 * e + 1] = (int32_t)j;
    }
    if (!pp.empty() &&
        cudaMemcpy(const_cast<int32_t*>(d.pairs), pp.data(), pp.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail_free(FTH_E_CUDA, "h2d pairs");
    if (cudaStreamSynchronize(P->stream) != cudaSuccess ||
        cudaMemcpy(P->d_desc + slot, &d, sizeof(PoolDesc), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail_free(FTH_E_CUDA, "h2d descriptor");
    P->probs[slot] = std::move(pr);
    P->dirty = true;
    *handle = slot;
    return FTH_OK;
}

fth_status fth_pool_remove(fth_pool* P, int64_t h) {
    if (!P || h < 0 || h >= (int64_t)P->probs.size() || !P->probs[h].used) return FTH_E_INVALID_ARG;
    PCK(cudaStreamSynchronize(P->stream), "sync");
    Problem& pr = P->probs[h];
    slab_free(P, pr.off, pr.bytes);
    pr = Problem();
    P->dirty = true;
    return FTH_OK;
}

fth_status fth_pool_run(fth_pool* P, int64_t steps) {
    if (!P || steps < 0) return FTH_E_INVALID_ARG;
    if (P->dirty) {
        const fth_status st = rebuild_lists(P);
        if (st != FTH_OK) return st;
    }
    if (P->h_live.empty() || steps == 0) return FTH_OK;
    // tune on the first run and again when the dense work list changed by over a quarter
    const bool drift = P->tuned && 4 * std::abs(P->n_force - P->tuned_items) > P->tuned_items;
    if ((!P->tuned || drift) && P->n_force > 0) {
        const fth_status st = autotune(P);
        if (st != FTH_OK) return st;
    }
    int64_t done = 0;
    if (!P->gle_tuned && P->n_dense_rows > 0 && steps >= kGleTuneSteps) {
        const fth_status st = autotune_gle(P);
        if (st != FTH_OK) return st;
        done = kGleTuneSteps;
    }
    if (P->graph_steps > 0 && steps - done >= P->graph_steps) {
        if (!P->graph_valid) {
            if (P->gexec) {
                cudaGraphExecDestroy(P->gexec);
                P->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            PCK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal), "capture");
            fth_status st = FTH_OK;
            for (int64_t k = 0; k < P->graph_steps && st == FTH_OK; ++k) st = enqueue_step(P);
            const cudaError_t ec = cudaStreamEndCapture(P->stream, &g);
            if (st != FTH_OK) return st;
            PCK(ec, "end capture");
            PCK(cudaGraphInstantiate(&P->gexec, g, 0), "graph instantiate");
            cudaGraphDestroy(g);
            P->graph_valid = true;
            ++P->graphs;
        }
        for (; done + P->graph_steps <= steps; done += P->graph_steps)
            PCK(cudaGraphLaunch(P->gexec, P->stream), "graph launch");
    }
    for (; done < steps; ++done) {
        const fth_status st = enqueue_step(P);
        if (st != FTH_OK) return st;
    }
    return FTH_OK;
}

fth_status fth_pool_profile(fth_pool* P, int64_t steps, double* ms, int64_t* launches) {
    if (!P || !ms || steps < 0) return FTH_E_INVALID_ARG;
    for (int c = 0; c < FTH_PK_CLASSES; ++c) {
        ms[c] = 0.0;
        if (launches) launches[c] = 0;
    }
    if (P->dirty) {
        const fth_status st = rebuild_lists(P);
        if (st != FTH_OK) return st;
    }
    if (P->h_live.empty()) return FTH_OK;
    cudaEvent_t ev[2 * FTH_PK_CLASSES];
    for (auto& e : ev) PCK(cudaEventCreate(&e), "event");
    const bool has[FTH_PK_CLASSES] = {P->n_force > 0, P->n_dense_rows > 0, P->n_csr_rows > 0, true};
    fth_status st = FTH_OK;
    for (int64_t k = 0; k < steps && st == FTH_OK; ++k) {
        st = enqueue_step(P, ev);
        if (st == FTH_OK && cudaStreamSynchronize(P->stream) != cudaSuccess)
            st = perr(P, FTH_E_CUDA, "sync");
        for (int c = 0; c < FTH_PK_CLASSES && st == FTH_OK; ++c) {
            if (!has[c]) continue;
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[2 * c], ev[2 * c + 1]);
            ms[c] += t;
            if (launches) ++launches[c];
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return st;
}

fth_status fth_pool_progress(fth_pool* P, double* rel_err, int64_t* blocks) {
    if (!P || !rel_err) return FTH_E_INVALID_ARG;
    if (P->dirty) {
        const fth_status st = rebuild_lists(P);
        if (st != FTH_OK) return st;
    }
    const int64_t nslot = P->max_problems;
    for (int64_t h = 0; h < nslot; ++h) {
        rel_err[h] = NAN;
        if (blocks) blocks[h] = -1;
    }
    if (P->h_live.empty()) return FTH_OK;
    std::vector<double> buf((size_t)nslot * 2);
    PCK(launch_pool_progress(P->d_desc, P->d_live, (int)P->h_live.size(), P->d_prog, P->stream),
        "progress");
    PCK(cudaMemcpyAsync(buf.data(), P->d_prog, buf.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        P->stream), "d2h progress");
    PCK(cudaStreamSynchronize(P->stream), "sync");
    for (int h : P->h_live) {
        rel_err[h] = buf[2 * (size_t)h];
        if (blocks) blocks[h] = (int64_t)buf[2 * (size_t)h + 1];
    }
    return FTH_OK;
}

fth_status fth_pool_get_state(fth_pool* P, int64_t h, int plane, double* host) {
    if (!P || !host || h < 0 || h >= (int64_t)P->probs.size() || !P->probs[h].used)
        return FTH_E_INVALID_ARG;
    if (plane != FTH_PLANE_Q && plane != FTH_PLANE_P && plane != FTH_PLANE_S) return FTH_E_INVALID_ARG;
    PoolDesc d;
    PCK(cudaStreamSynchronize(P->stream), "sync");
    PCK(cudaMemcpy(&d, P->d_desc + h, sizeof d, cudaMemcpyDeviceToHost), "d2h descriptor");
    const int64_t n = d.n, R = P->R, na = plane == FTH_PLANE_S ? d.ns - 1 : 1;
    if (na < 1) return FTH_OK;
    const float* src = plane == FTH_PLANE_Q ? d.q[d.cur] : plane == FTH_PLANE_P ? d.p : d.s;
    std::vector<float> buf((size_t)(na * n * R));
    PCK(cudaMemcpy(buf.data(), src, buf.size() * 4, cudaMemcpyDeviceToHost), "d2h state");
    for (int64_t a = 0; a < na; ++a)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t r = 0; r < R; ++r)
                host[(r * na + a) * n + i] = buf[(size_t)((a * n + i) * R + r)];
    return FTH_OK;
}

fth_status fth_pool_problem_info(fth_pool* P, int64_t h, fth_info_t* info) {
    if (!P || !info || h < 0 || h >= (int64_t)P->probs.size() || !P->probs[h].used)
        return FTH_E_INVALID_ARG;
    PoolDesc d;
    PCK(cudaStreamSynchronize(P->stream), "sync");
    PCK(cudaMemcpy(&d, P->d_desc + h, sizeof d, cudaMemcpyDeviceToHost), "d2h descriptor");
    std::memset(info, 0, sizeof *info);
    info->steps = d.t;
    info->samples = d.nsamp;
    info->accumulated = d.nblocks * d.block + d.inblock;
    info->blocks = d.nblocks;
    info->primed = d.primed;
    info->precision = d.kind == 0 ? P->prec : FTH_PREC_FP32;
    info->n = d.n;
    info->replicas = P->R;
    info->tracked = d.npairs;
    info->workspace_bytes = P->probs[h].bytes;
    return FTH_OK;
}

fth_status fth_pool_elements(fth_pool* P, int64_t h, const int64_t* pairs, int64_t k,
                             double* values, double* errbars) {
    if (!P || h < 0 || h >= (int64_t)P->probs.size() || !P->probs[h].used) return FTH_E_INVALID_ARG;
    if (k < 0 || (k > 0 && (!pairs || !values))) return FTH_E_INVALID_ARG;
    const Problem& pr = P->probs[h];
    PoolDesc d;
    PCK(cudaStreamSynchronize(P->stream), "sync");
    uint32_t e = 0;
    PCK(cudaMemcpy(&e, P->d_err, 4, cudaMemcpyDeviceToHost), "d2h err");
    if (e & kErrTimeout) return perr(P, FTH_E_TIMEOUT, "a device wait timed out");
    if (e & kErrNonFinite) return perr(P, FTH_E_NONFINITE, "non-finite accumulator");
    PCK(cudaMemcpy(&d, P->d_desc + h, sizeof d, cudaMemcpyDeviceToHost), "d2h descriptor");
    const int64_t np = pr.npairs;
    std::vector<double> mean(np), m2(np);
    std::vector<float> part(np);
    if (np) {
        PCK(cudaMemcpy(mean.data(), d.mean, np * 8, cudaMemcpyDeviceToHost), "d2h mean");
        PCK(cudaMemcpy(m2.data(), d.m2, np * 8, cudaMemcpyDeviceToHost), "d2h m2");
        PCK(cudaMemcpy(part.data(), d.partial, np * 4, cudaMemcpyDeviceToHost), "d2h partial");
    }
    const double nb = (double)d.nblocks, R = (double)P->R;
    const double nacc = (double)(d.nblocks * d.block + d.inblock);
    for (int64_t q = 0; q < k; ++q) {
        auto it = pr.pair_index.find(pkey(pairs[2 * q], pairs[2 * q + 1]));
        if (it == pr.pair_index.end()) return perr(P, FTH_E_NOT_TRACKED, "element not tracked");
        const int64_t x = it->second;
        const double total = mean[x] * nb * (double)d.block * R + (double)part[x];
        values[q] = nacc > 0 ? total / (nacc * R) : NAN;
        if (errbars) errbars[q] = nb >= 2 ? std::sqrt(m2[x] / (nb * (nb - 1.0))) : NAN;
    }
    return FTH_OK;
}

fth_status fth_pool_stats(const fth_pool* P, fth_pool_stats_t* s) {
    if (!P || !s) return FTH_E_INVALID_ARG;
    s->live = 0;
    for (const auto& pr : P->probs) s->live += pr.used ? 1 : 0;
    s->slab_bytes = P->slab_end - P->slab_begin;
    s->used_bytes = P->used_bytes;
    s->force_items = P->n_force;
    s->gle_items = P->n_dense_rows;
    s->csr_items = P->n_csr_rows;
    s->tuned_variant = P->variant;
    s->tuned_grid = P->grid;
    s->tuned_us = P->tuned_us;
    s->gle_variant = P->gle_variant;
    s->gle_us = P->gle_us;
    s->graphs = P->graphs;
    return FTH_OK;
}

const char* fth_pool_last_error(const fth_pool* P) { return P ? P->last_error.c_str() : ""; }

void fth_pool_destroy(fth_pool* P) {
    if (!P) return;
    if (P->stream) cudaStreamSynchronize(P->stream);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    delete P;
}

}  // extern "C"
