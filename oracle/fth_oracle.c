/*
 * CPU oracle for the f-thermostat (FTH) hot path.  TEST INFRASTRUCTURE ONLY:
 * it is loaded by the tests, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg, never by the library.  Plain, slow FP64 loops; nothing here is
 * shared with the CUDA path.
 *
 * What it computes (paper: Nava, Ceriotti, Dryzun, Parrinello, "Evaluating
 * functions of positive-definite matrices using colored noise thermostats"):
 *   - the harmonic force F = -M q of the potential V = q^T M q / 2 (Eq. 5);
 *   - the Markovian GLE of Eq. 2 on every Cartesian dof, integrated with the
 *     modified velocity Verlet scheme the paper cites (Sec. "The f-thermostat"):
 *     per step  O(dt/2) B(dt/2) A(dt) [force] B(dt/2) O(dt/2), where the O
 *     half-step is the exact Ornstein-Uhlenbeck update of (p, s):
 *     p~ <- T p~ + S xi, T = exp(-A_p dt/2), S S^T = C_p - T C_p T^T (Eq. 4);
 *   - samples of p (or q) at the end of each step and their running
 *     second moments <x_i x_j> (Eq. 6), block averaged for error bars
 *     (Sec. "Results and benchmarks", memory-footprint paragraph).
 *
 * Noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) written from its
 * published definition, and the Box-Muller transform.  Replicas are paired: for
 * "kick index" kappa, dof i and replica pair j, Philox call k uses counter
 * (kappa, i, j, k) and key (seed_lo, seed_hi), and the calls k = 0, 1, ... form one
 * stream of normals, four per call.  Each uint32 pair (x0,x1) gives two of them:
 *   u(x) = ((x >> 9) * 2 + 1) * 2^-24,  rho = sqrt(-2 ln u(x0)),
 *   n0 = rho cos(2 pi u(x1)),  n1 = rho sin(2 pi u(x1)).
 * Replica r (global index r + roff, roff: global index of the first replica) belongs
 * to pair j = (r + roff) / 2 and takes the stream positions h W .. h W + W - 1,
 * h = (r + roff) mod 2, W = ns + 1 (the normals one fused launch needs); so 2W normals
 * per pair use all four words of ceil(2W / 4) calls.
 *
 * The two O half-steps of a fused launch (ending step kappa-1 and starting step
 * kappa) are separated only by the end-of-step sample, which observes p after the
 * first one.  They are drawn jointly from their exact joint law: with v the state
 * after the end-of-step kick, the sample is (T v)_0 + x and the next state is
 * T^2 v + y, where (x, y) = L zeta, zeta = normals 0..ns of kappa, and L L^T is the
 * covariance of (x, y) = (e_0^T S xi1, T S xi1 + S xi2) -- the same Markov chain as
 * two independent half-steps, with ns + 1 normals instead of 2 ns.  The prologue
 * (start half only) uses normals 0..ns-1 of its kappa for a single O half-step.
 *
 * State layout: q[R][n], p[R][n], s[R][ns-1][n]  (replica-major).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NS_MAX 8

/* ---------------------------------------------------------------- Philox */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

static double unit_open(uint32_t x)
{
    return (double)((x >> 9) * 2u + 1u) * (1.0 / 16777216.0);
}

/* `count` normals for (kappa, i, r); count <= 4 * ceil(2*NS_MAX/4). */
void oracle_normals(uint64_t seed, uint32_t kappa, uint32_t i, uint32_t r, int count, double* out)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; 4 * k < count; ++k) {
        const uint32_t ctr[4] = {kappa, i, r, (uint32_t)k};
        uint32_t x[4];
        oracle_philox4x32_10(ctr, key, x);
        for (int h = 0; h < 2; ++h) {
            const double rho = sqrt(-2.0 * log(unit_open(x[2 * h])));
            const double th = two_pi * unit_open(x[2 * h + 1]);
            const int j = 4 * k + 2 * h;
            if (j < count) out[j] = rho * cos(th);
            if (j + 1 < count) out[j + 1] = rho * sin(th);
        }
    }
}

/* The first `count` (<= width) normals of global replica r: stream positions
 * (r mod 2) * width + t of the pair stream of j = r / 2. */
void oracle_replica_normals(uint64_t seed, uint32_t kappa, uint32_t i, uint32_t r, int width,
                            int count, double* out)
{
    double buf[4 * ((2 * (NS_MAX + 1) + 3) / 4)];
    const int need = 4 * ((2 * width + 3) / 4);
    oracle_normals(seed, kappa, i, r >> 1, need, buf);
    const int h0 = (int)(r & 1u) * width;
    for (int t = 0; t < count; ++t) out[t] = buf[h0 + t];
}

/* ---------------------------------------------------------------- force */
/* F[r][i] = -(M q_r)_i.  kind 0: dense row-major n x n; kind 1: CSR. */
static void force(int64_t n, int64_t R, int kind, const double* Md, const int64_t* rowptr,
                  const int64_t* col, const double* val, const double* q, double* F)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < R; ++r) {
        const double* qr = q + r * n;
        double* Fr = F + r * n;
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            if (kind == 0) {
                const double* mi = Md + i * n;
                for (int64_t k = 0; k < n; ++k) acc += mi[k] * qr[k];
            } else {
                for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) acc += val[e] * qr[col[e]];
            }
            Fr[i] = -acc;
        }
    }
}

/* p~ <- T p~ + S xi on one (r, i): v[0] = p, v[1..ns-1] = s. */
static void o_half(int ns, const double* T, const double* S, double* v, const double* xi)
{
    double out[NS_MAX];
    for (int a = 0; a < ns; ++a) {
        double acc = 0.0;
        for (int b = 0; b < ns; ++b) acc += T[a * ns + b] * v[b];
        for (int b = 0; b <= a; ++b) acc += S[a * ns + b] * xi[b];
        out[a] = acc;
    }
    for (int a = 0; a < ns; ++a) v[a] = out[a];
}

static void load_v(int64_t n, int ns, int64_t r, int64_t i, const double* p, const double* s, double* v)
{
    v[0] = p[r * n + i];
    for (int a = 1; a < ns; ++a) v[a] = s[(r * (ns - 1) + (a - 1)) * n + i];
}

static void store_v(int64_t n, int ns, int64_t r, int64_t i, double* p, double* s, const double* v)
{
    p[r * n + i] = v[0];
    for (int a = 1; a < ns; ++a) s[(r * (ns - 1) + (a - 1)) * n + i] = v[a];
}

/* Start half of the step with kick index kappa: O(dt/2) B(dt/2) A(dt). */
int oracle_prologue(int64_t n, int64_t R, int ns, int kind, const double* Md,
                    const int64_t* rowptr, const int64_t* col, const double* val,
                    const double* T, const double* S, double dt, uint64_t seed,
                    uint32_t roff, uint32_t kappa, double* q, double* p, double* s)
{
    if (ns < 1 || ns > NS_MAX) return -1;
    double* F = (double*)malloc(sizeof(double) * (size_t)(n * R));
    if (!F) return -2;
    force(n, R, kind, Md, rowptr, col, val, q, F);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < R; ++r) {
        double xi[2 * NS_MAX], v[NS_MAX];
        for (int64_t i = 0; i < n; ++i) {
            oracle_replica_normals(seed, kappa, (uint32_t)i, (uint32_t)r + roff, ns + 1, ns, xi);
            load_v(n, ns, r, i, p, s, v);
            o_half(ns, T, S, v, xi);
            v[0] += 0.5 * dt * F[r * n + i];
            store_v(n, ns, r, i, p, s, v);
            q[r * n + i] += dt * v[0];
        }
    }
    free(F);
    return 0;
}

/*
 * `nsteps` fused step pairs.  Launch j (kick index kappa0 + j) computes the force at
 * the current positions, finishes the current step (B, O, sample) and starts the
 * next one (O, B, A).  Samples are written to `samples` ([nsteps][R][n]) when it is
 * non-NULL.  T2 = T T ([ns][ns]) and Lj ([ns+1][ns+1], lower) give the joint O
 * half-steps described at the top of this file.
 *
 * Accumulation over the tracked pairs (i, j) of x = p (observable 0) or q (1):
 *   nsamp      samples seen so far (burn-in included); samples with index < burnin
 *              are discarded;
 *   partial    per pair, sum over the current block of sum_r x_i x_j;
 *   inblock    samples in the current block;
 *   nblocks, bmean, bm2   Welford mean and M2 of the completed block means, where
 *              a block mean is partial / (block * R).
 */
int oracle_steps(int64_t n, int64_t R, int ns, int kind, const double* Md,
                 const int64_t* rowptr, const int64_t* col, const double* val,
                 const double* T, const double* S, const double* T2, const double* Lj,
                 double dt, uint64_t seed,
                 uint32_t roff, uint32_t kappa0, int64_t nsteps, double* q, double* p, double* s,
                 int observable, double* samples,
                 int64_t npairs, const int64_t* pairs, int64_t burnin, int64_t block,
                 int64_t* nsamp, double* partial, int64_t* inblock,
                 int64_t* nblocks, double* bmean, double* bm2)
{
    if (ns < 1 || ns > NS_MAX) return -1;
    double* F = (double*)malloc(sizeof(double) * (size_t)(n * R));
    double* X = (double*)malloc(sizeof(double) * (size_t)(n * R));
    if (!F || !X) {
        free(F);
        free(X);
        return -2;
    }
    for (int64_t step = 0; step < nsteps; ++step) {
        const uint32_t kappa = kappa0 + (uint32_t)step;
        force(n, R, kind, Md, rowptr, col, val, q, F);
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < R; ++r) {
            double zeta[NS_MAX + 4], v[NS_MAX], out[NS_MAX];
            const int m = ns + 1;
            for (int64_t i = 0; i < n; ++i) {
                const double f = F[r * n + i];
                oracle_replica_normals(seed, kappa, (uint32_t)i, (uint32_t)r + roff, m, m, zeta);
                load_v(n, ns, r, i, p, s, v);
                v[0] += 0.5 * dt * f;          /* B(dt/2), end of the current step */
                /* p after the end-of-step O(dt/2): (T v)_0 + x, x = (L zeta)_0 */
                double pmid = Lj[0] * zeta[0];
                for (int b = 0; b < ns; ++b) pmid += T[b] * v[b];
                X[r * n + i] = observable ? q[r * n + i] : pmid;
                /* both O(dt/2): T^2 v + y, y = (L zeta)_1..ns */
                for (int a = 0; a < ns; ++a) {
                    double acc = 0.0;
                    for (int b = 0; b < ns; ++b) acc += T2[a * ns + b] * v[b];
                    for (int b = 0; b <= a + 1; ++b) acc += Lj[(a + 1) * m + b] * zeta[b];
                    out[a] = acc;
                }
                for (int a = 0; a < ns; ++a) v[a] = out[a];
                v[0] += 0.5 * dt * f;          /* B(dt/2) */
                store_v(n, ns, r, i, p, s, v);
                q[r * n + i] += dt * v[0];     /* A(dt) */
            }
        }
        if (samples) memcpy(samples + step * n * R, X, sizeof(double) * (size_t)(n * R));
        if (npairs > 0 && *nsamp >= burnin) {
#pragma omp parallel for schedule(static)
            for (int64_t e = 0; e < npairs; ++e) {
                const int64_t i = pairs[2 * e], j = pairs[2 * e + 1];
                double acc = 0.0;
                for (int64_t r = 0; r < R; ++r) acc += X[r * n + i] * X[r * n + j];
                partial[e] += acc;
            }
            *inblock += 1;
            if (*inblock == block) {
                *nblocks += 1;
                const double nb = (double)*nblocks;
                for (int64_t e = 0; e < npairs; ++e) {
                    const double b = partial[e] / ((double)block * (double)R);
                    const double d = b - bmean[e];
                    bmean[e] += d / nb;
                    bm2[e] += d * (b - bmean[e]);
                    partial[e] = 0.0;
                }
                *inblock = 0;
            }
        }
        *nsamp += 1;
    }
    free(F);
    free(X);
    return 0;
}

/* Exposed for tests: F = -M q for a single replica set. */
void oracle_force(int64_t n, int64_t R, int kind, const double* Md, const int64_t* rowptr,
                  const int64_t* col, const double* val, const double* q, double* F)
{
    force(n, R, kind, Md, rowptr, col, val, q, F);
}
