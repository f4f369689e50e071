// Serving loop over a problem pool: requests (a matrix, a GLE, tracked elements, an
// accuracy target) arrive at any time, wait in a queue, are admitted into the pool as
// soon as a slot and enough workspace are free (admission by device footprint), are
// stepped together with everything else on the device (continuous batching), and are
// retired as soon as the normwise relative error bar of their tracked elements meets
// their target or their step budget is spent.  A request's result does not depend on
// what else is in the pool: its noise key is its own seed and the pool's arithmetic
// per problem is independent of the mix.
//
// The estimate of f(M)_ij is the paper's Eq. 6 (average of p_i p_j over replicas and
// time, block-averaged for the error bar); the retire rule is the error bar of that
// average against the requested relative accuracy.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "fth.h"

namespace {

struct Request {
    int64_t id = -1;
    int state = FTH_REQ_QUEUED;
    // host copies of the inputs (kept until admitted)
    fth_matrix M{};
    std::vector<uint8_t> values;
    std::vector<int32_t> rowptr, colind;
    fth_gle gle{};
    fth_problem_options po{};
    std::vector<int64_t> pairs;
    double target = 0.0;
    int64_t max_steps = 0;
    // progress and result
    int64_t handle = -1;
    int64_t steps_at_admit = 0;   // server step counter when admitted
    int64_t steps = 0;            // steps this request ran
    double rel_err = NAN;
    std::vector<double> values_out, errbars_out;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    int64_t bypassed = 0;         // admissions of later requests while this one waited
};

}  // namespace

struct fth_server {
    fth_pool* pool = nullptr;
    int64_t max_problems = 0;
    int64_t chunk_steps = 0;
    int64_t min_blocks = 2;
    int64_t max_bypass = 0;
    int64_t steps = 0;            // server steps so far
    std::deque<Request> reqs;     // by id (stable addresses: inputs point into them)
    std::deque<int64_t> queue;    // ids waiting for admission, arrival order
    std::vector<int64_t> running; // ids in the pool
    std::vector<double> rel;
    std::vector<int64_t> blocks;
    std::chrono::steady_clock::time_point t0;
    std::string last_error;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

fth_status serr(fth_server* S, fth_status st, const std::string& m) {
    if (S) S->last_error = m;
    return st;
}

// Try to admit queued requests in arrival order; a request that does not fit is skipped
// (later, smaller ones may fit) unless it has already been bypassed max_bypass times,
// in which case admission stops until it fits (no starvation).
fth_status admit(fth_server* S, int64_t* admitted) {
    *admitted = 0;
    for (auto it = S->queue.begin(); it != S->queue.end();) {
        Request& r = S->reqs[*it];
        int64_t h = -1;
        const fth_status st = fth_pool_add(S->pool, &r.M, &r.gle, &r.po, &h);
        if (st == FTH_OK) {
            r.handle = h;
            r.state = FTH_REQ_RUNNING;
            r.steps_at_admit = S->steps;
            r.t_admit = S->now();
            // the inputs now live on the device
            std::vector<uint8_t>().swap(r.values);
            std::vector<int32_t>().swap(r.rowptr);
            std::vector<int32_t>().swap(r.colind);
            S->running.push_back(r.id);
            ++*admitted;
            for (auto jt = S->queue.begin(); jt != it; ++jt) ++S->reqs[*jt].bypassed;
            it = S->queue.erase(it);
            continue;
        }
        bool never_fits = false;
        if (st == FTH_E_WORKSPACE) {
            // a request larger than the whole slab would block the queue for ever
            size_t need = 0;
            fth_pool_stats_t ps;
            never_fits = fth_pool_footprint(S->pool, &r.M, &r.gle, &r.po, &need) == FTH_OK &&
                         fth_pool_stats(S->pool, &ps) == FTH_OK && need > ps.slab_bytes;
        }
        if (st != FTH_E_WORKSPACE || never_fits) {
            // invalid (or never admissible) request: finish it, keep serving the others
            r.state = FTH_REQ_FAILED;
            r.t_done = S->now();
            S->last_error = never_fits ? std::string("request larger than the pool's workspace")
                                       : std::string(fth_pool_last_error(S->pool));
            it = S->queue.erase(it);
            continue;
        }
        if (r.bypassed >= S->max_bypass) break;
        ++it;
    }
    return FTH_OK;
}

fth_status retire(fth_server* S, int64_t* retired) {
    *retired = 0;
    if (S->running.empty()) return FTH_OK;
    fth_status st = fth_pool_progress(S->pool, S->rel.data(), S->blocks.data());
    if (st != FTH_OK) return serr(S, st, fth_pool_last_error(S->pool));
    std::vector<int64_t> keep;
    for (int64_t id : S->running) {
        Request& r = S->reqs[id];
        r.steps = S->steps - r.steps_at_admit;
        r.rel_err = S->rel[r.handle];
        const bool met = S->blocks[r.handle] >= S->min_blocks && r.rel_err <= r.target;
        const bool spent = r.max_steps > 0 && r.steps >= r.max_steps;
        if (!met && !spent) {
            keep.push_back(id);
            continue;
        }
        const int64_t k = (int64_t)r.pairs.size() / 2;
        r.values_out.assign(k, NAN);
        r.errbars_out.assign(k, NAN);
        st = fth_pool_elements(S->pool, r.handle, r.pairs.data(), k, r.values_out.data(),
                               r.errbars_out.data());
        if (st != FTH_OK) return serr(S, st, fth_pool_last_error(S->pool));
        st = fth_pool_remove(S->pool, r.handle);
        if (st != FTH_OK) return serr(S, st, fth_pool_last_error(S->pool));
        r.handle = -1;
        r.state = met ? FTH_REQ_DONE : FTH_REQ_BUDGET;
        r.t_done = S->now();
        ++*retired;
    }
    S->running.swap(keep);
    return FTH_OK;
}

}  // namespace

extern "C" {

fth_status fth_server_create(const fth_server_options* opt, void* workspace, size_t bytes,
                             fth_server** out) {
    if (!opt || !out || opt->chunk_steps < 1 || opt->min_blocks < 2 || opt->max_bypass < 0)
        return FTH_E_INVALID_ARG;
    *out = nullptr;
    fth_pool* pool = nullptr;
    const fth_status st = fth_pool_create(&opt->pool, workspace, bytes, &pool);
    if (st != FTH_OK) return st;
    fth_server* S = new fth_server();
    S->pool = pool;
    S->max_problems = opt->pool.max_problems;
    S->chunk_steps = opt->chunk_steps;
    S->min_blocks = opt->min_blocks;
    S->max_bypass = opt->max_bypass;
    S->rel.assign((size_t)S->max_problems, NAN);
    S->blocks.assign((size_t)S->max_problems, -1);
    S->t0 = std::chrono::steady_clock::now();
    *out = S;
    return FTH_OK;
}

fth_status fth_server_submit(fth_server* S, const fth_matrix* M, const fth_gle* gle,
                             const fth_problem_options* po, double target, int64_t max_steps,
                             int64_t* id) {
    if (!S || !M || !gle || !po || !id || !M->values || M->n < 1) return FTH_E_INVALID_ARG;
    if (!(target > 0.0) || max_steps < 0 || po->npairs < 1 || !po->pairs) return FTH_E_INVALID_ARG;
    if (M->kind != FTH_DENSE && M->kind != FTH_CSR) return FTH_E_INVALID_ARG;
    if (M->dtype != FTH_F32 && M->dtype != FTH_F64) return FTH_E_INVALID_ARG;
    Request r;
    r.id = (int64_t)S->reqs.size();
    r.M = *M;
    const size_t esz = M->dtype == FTH_F64 ? 8 : 4;
    const size_t nvals = M->kind == FTH_DENSE ? (size_t)M->n * M->n : (size_t)M->nnz;
    r.values.resize(std::max<size_t>(nvals * esz, 1));
    auto fetch = [&](void* dst, const void* src, size_t b) {
        if (!b) return true;
        if (M->on_device) return cudaMemcpy(dst, src, b, cudaMemcpyDeviceToHost) == cudaSuccess;
        std::memcpy(dst, src, b);
        return true;
    };
    if (!fetch(r.values.data(), M->values, nvals * esz)) return serr(S, FTH_E_CUDA, "copy M");
    if (M->kind == FTH_CSR) {
        if (!M->rowptr || !M->colind) return FTH_E_INVALID_ARG;
        r.rowptr.resize((size_t)M->n + 1);
        r.colind.resize(std::max<size_t>((size_t)M->nnz, 1));
        if (!fetch(r.rowptr.data(), M->rowptr, r.rowptr.size() * 4) ||
            !fetch(r.colind.data(), M->colind, (size_t)M->nnz * 4))
            return serr(S, FTH_E_CUDA, "copy CSR");
        r.M.rowptr = r.rowptr.data();
        r.M.colind = r.colind.data();
    }
    r.M.values = r.values.data();
    r.M.on_device = 0;
    r.gle = *gle;
    r.po = *po;
    r.pairs.assign(po->pairs, po->pairs + 2 * po->npairs);
    r.po.pairs = r.pairs.data();
    r.target = target;
    r.max_steps = max_steps;
    r.t_submit = S->now();
    S->reqs.push_back(std::move(r));
    Request& q = S->reqs.back();
    // point the pool inputs at the request's own copies
    q.M.values = q.values.data();
    if (q.M.kind == FTH_CSR) {
        q.M.rowptr = q.rowptr.data();
        q.M.colind = q.colind.data();
    }
    q.po.pairs = q.pairs.data();
    S->queue.push_back(q.id);
    *id = q.id;
    return FTH_OK;
}

fth_status fth_server_step(fth_server* S, fth_server_counts* c) {
    if (!S) return FTH_E_INVALID_ARG;
    int64_t admitted = 0, retired = 0;
    fth_status st = admit(S, &admitted);
    if (st != FTH_OK) return st;
    if (!S->running.empty()) {
        st = fth_pool_run(S->pool, S->chunk_steps);
        if (st != FTH_OK) return serr(S, st, fth_pool_last_error(S->pool));
        S->steps += S->chunk_steps;
        st = retire(S, &retired);
        if (st != FTH_OK) return st;
    }
    if (c) {
        c->admitted = admitted;
        c->retired = retired;
        c->running = (int64_t)S->running.size();
        c->queued = (int64_t)S->queue.size();
        c->steps = S->steps;
        fth_pool_stats_t ps;
        fth_pool_stats(S->pool, &ps);
        c->used_bytes = ps.used_bytes;
        c->slab_bytes = ps.slab_bytes;
    }
    return FTH_OK;
}

fth_status fth_server_result(fth_server* S, int64_t id, fth_request_info* info, double* values,
                             double* errbars) {
    if (!S || !info || id < 0 || id >= (int64_t)S->reqs.size()) return FTH_E_INVALID_ARG;
    const Request& r = S->reqs[id];
    info->state = r.state;
    info->steps = r.state == FTH_REQ_RUNNING ? S->steps - r.steps_at_admit : r.steps;
    info->rel_err = r.rel_err;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
    info->npairs = (int64_t)r.pairs.size() / 2;
    if ((r.state == FTH_REQ_DONE || r.state == FTH_REQ_BUDGET) && values) {
        std::memcpy(values, r.values_out.data(), r.values_out.size() * sizeof(double));
        if (errbars) std::memcpy(errbars, r.errbars_out.data(), r.errbars_out.size() * sizeof(double));
    }
    return FTH_OK;
}

double fth_server_clock(const fth_server* S) { return S ? S->now() : 0.0; }

fth_pool* fth_server_pool(fth_server* S) { return S ? S->pool : nullptr; }

const char* fth_server_last_error(const fth_server* S) { return S ? S->last_error.c_str() : ""; }

void fth_server_destroy(fth_server* S) {
    if (!S) return;
    fth_pool_destroy(S->pool);
    delete S;
}

}  // extern "C"
