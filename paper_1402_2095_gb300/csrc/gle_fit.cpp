// Host-side GLE fitter and per-mode response (FP64): fth_fit_gle, fth_gle_response.
//
// The f-thermostat needs a GLE whose normal mode of frequency w has momentum
// fluctuations <p^2>(w) = f(w^2) over the spectrum of M (Sec. "The f-thermostat", the
// fitting paragraph; Eq. 2 and Eq. 4).  The paper fits the drift A_p and the
// free-particle covariance C_p by least squares, starting from delta-like memory kernels
// and then refining the general form, and asks of a fit (Sec. "Results and
// benchmarks") that it (1) follows f over the spectral range, (2) may be only an upper
// bound where f is below a small threshold (the exponential-tail rule), and (3) keeps the
// correlation times short, since the statistical error grows with them.
//
// What is fitted here is the response of the integrator actually run, at the time step
// actually used: per mode, the stationary covariance of the sample-to-sample map of the
// velocity Verlet GLE step (the paper notes that fitting for a given time step corrects
// the finite-dt error).  For one mode of eigenvalue lam the state x = (q, p, s_1..s_s)
// evolves linearly, x' = G x + noise with covariance Qn (O = diag(1, T), Sig = [0; S],
// V = B A B, B = I - (lam dt/2) e_p e_q^T, A = I + dt e_q e_p^T, G = O V O,
// Qn = (O V Sig)(O V Sig)^T + Sig Sig^T), and C = G C G^T + Qn is solved directly on the
// d (d + 1) / 2 distinct entries of the symmetric C.
//
// Parametrisation: A_p = L L^T + W (L lower triangular with exp'd diagonal, W skew), so
// every eigenvalue of A_p has a positive real part; the diffusion B_p B_p^T with B_p lower
// triangular; C_p solves A_p C_p + C_p A_p^T = B_p B_p^T (Eq. 4), so it is a valid
// covariance.  The overall scale gamma of C_p (the response is linear in it) is solved in
// closed form at every evaluation.  Optimiser: Levenberg-Marquardt with a forward-
// difference Jacobian, several seeded starts (run on host threads) whose auxiliary
// block holds damped oscillators spread over the frequency range (the delta-like start).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

#include "fth.h"

namespace {

constexpr int kMaxNs = 5;               // (p, s_1..s_4)
constexpr int kMaxD = kMaxNs + 1;       // (q, p, s_1..s_4)
constexpr int kMaxSym = kMaxD * (kMaxD + 1) / 2;
constexpr double kBad = 1e3;            // residual of an invalid parameter point

// ------------------------------------------------------------------ small dense algebra
// In-place LU with partial pivoting of the n x n row-major A; false if singular.
bool lu_factor(int n, double* A, int* piv) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(A[i * n + k]) > best) {
                best = std::fabs(A[i * n + k]);
                p = i;
            }
        if (!(best > 0.0) || !std::isfinite(best)) return false;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
        const double inv = 1.0 / A[k * n + k];
        for (int i = k + 1; i < n; ++i) {
            const double l = A[i * n + k] * inv;
            A[i * n + k] = l;
            if (l != 0.0)
                for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return true;
}

// Solve with the factors of lu_factor: the row swaps were applied to whole rows (the
// stored multipliers included), so all of them act on b before the forward sweep.
void lu_solve(int n, const double* LU, const int* piv, double* b) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int k = 0; k < n; ++k)
        for (int i = k + 1; i < n; ++i) b[i] -= LU[i * n + k] * b[k];
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= LU[i * n + j] * b[j];
        b[i] = s / LU[i * n + i];
    }
}

// c = a b for n x n row-major matrices.
void matmul(int n, const double* a, const double* b, double* c) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + j];
            c[i * n + j] = s;
        }
}

// Cholesky of the SPD n x n A (lower L in place); false if not positive definite.
bool cholesky(int n, double* A) {
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = s / d;
        }
        for (int k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
    }
    return true;
}

void chol_solve(int n, const double* L, double* b) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * b[k];
        b[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * b[k];
        b[i] = s / L[i * n + i];
    }
}

// ------------------------------------------------------------------ per-mode chain
// G and Qn of the sample-to-sample map of one mode (see the file header).
void mode_chain(int ns, const double* T, const double* S, double dt, double lam, double* G,
                double* Qn) {
    const int d = ns + 1;
    double O[kMaxD * kMaxD] = {}, V[kMaxD * kMaxD], Bm[kMaxD * kMaxD] = {}, Am[kMaxD * kMaxD] = {};
    double tmp[kMaxD * kMaxD];
    O[0] = 1.0;
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) O[(i + 1) * d + j + 1] = T[i * ns + j];
    for (int i = 0; i < d; ++i) Bm[i * d + i] = Am[i * d + i] = 1.0;
    Bm[1 * d + 0] = -0.5 * dt * lam;        // p <- p - (dt/2) lam q
    Am[0 * d + 1] = dt;                     // q <- q + dt p
    matmul(d, Bm, Am, tmp);
    matmul(d, tmp, Bm, V);
    double OV[kMaxD * kMaxD];
    matmul(d, O, V, OV);
    matmul(d, OV, O, G);
    // OVSig = OV[:, 1:] S  (d x ns);  Qn = OVSig OVSig^T + Sig Sig^T
    double OVS[kMaxD * kMaxNs];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < ns; ++j) {
            double s = 0.0;
            for (int k = 0; k < ns; ++k) s += OV[i * d + k + 1] * S[k * ns + j];
            OVS[i * ns + j] = s;
        }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < ns; ++k) s += OVS[i * ns + k] * OVS[j * ns + k];
            if (i > 0 && j > 0)
                for (int k = 0; k < ns; ++k) s += S[(i - 1) * ns + k] * S[(j - 1) * ns + k];
            Qn[i * d + j] = s;
        }
}

// Stationary second moment g = C[x][x] of the observable x (p: 1, q: 0) and the
// integrated correlation time of x^2 in samples, tau = 1 + 2 sum_{l>=1} rho(l)^2
// = (2 X_xx - g^2) / g^2 with X = G X G^T + (C e_x)(C e_x)^T (Gaussian chain:
// the autocovariance of x^2 at lag l is 2 c(l)^2, c(l) = e_x^T G^l C e_x).
bool mode_moments(int d, const double* G, const double* Qn, int x, double* g, double* tau) {
    const int m = d * (d + 1) / 2;
    int idx[kMaxD][kMaxD];
    int ia[kMaxSym], ib[kMaxSym];
    for (int i = 0, k = 0; i < d; ++i)
        for (int j = i; j < d; ++j, ++k) {
            idx[i][j] = idx[j][i] = k;
            ia[k] = i;
            ib[k] = j;
        }
    double K[kMaxSym * kMaxSym];
    int piv[kMaxSym];
    for (int r = 0; r < m; ++r) {
        const int i = ia[r], j = ib[r];
        for (int c = 0; c < m; ++c) {
            const int a = ia[c], b = ib[c];
            double v = G[i * d + a] * G[j * d + b];
            if (a != b) v += G[i * d + b] * G[j * d + a];
            K[r * m + c] = (r == c ? 1.0 : 0.0) - v;
        }
    }
    if (!lu_factor(m, K, piv)) return false;
    double c[kMaxSym];
    for (int r = 0; r < m; ++r) c[r] = Qn[ia[r] * d + ib[r]];
    lu_solve(m, K, piv, c);
    const double gx = c[idx[x][x]];
    if (!(gx > 0.0) || !std::isfinite(gx)) return false;
    *g = gx;
    if (tau) {
        double v[kMaxD];
        for (int i = 0; i < d; ++i) v[i] = c[idx[i][x]];
        double X[kMaxSym];
        for (int r = 0; r < m; ++r) X[r] = v[ia[r]] * v[ib[r]];
        lu_solve(m, K, piv, X);
        const double xx = X[idx[x][x]];
        *tau = (2.0 * xx - gx * gx) / (gx * gx);
        if (!std::isfinite(*tau)) return false;
    }
    return true;
}

// Continuous Lyapunov A C + C A^T = D for ns x ns matrices (Kronecker form); C symmetrised.
bool lyap_continuous(int ns, const double* A, const double* D, double* C) {
    const int m = ns * ns;
    std::vector<double> K((size_t)m * m, 0.0);
    std::vector<int> piv(m);
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) {
            const int r = i * ns + j;
            for (int k = 0; k < ns; ++k) {
                K[(size_t)r * m + k * ns + j] += A[i * ns + k];   // (A C)_ij
                K[(size_t)r * m + i * ns + k] += A[j * ns + k];   // (C A^T)_ij
            }
        }
    if (!lu_factor(m, K.data(), piv.data())) return false;
    double b[kMaxNs * kMaxNs];
    for (int r = 0; r < m; ++r) b[r] = D[r];
    lu_solve(m, K.data(), piv.data(), b);
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) C[i * ns + j] = 0.5 * (b[i * ns + j] + b[j * ns + i]);
    for (int r = 0; r < m; ++r)
        if (!std::isfinite(C[r])) return false;
    return true;
}

bool make_gle_struct(int ns, const double* a, const double* c, fth_gle* g) {
    std::memset(g, 0, sizeof *g);
    g->s = ns - 1;
    for (int k = 0; k < ns * ns; ++k) {
        g->a_p[k] = a[k];
        g->c_p[k] = c[k];
    }
    return true;
}

// Response g(lam) (and tau) of a GLE over a list of eigenvalues; false on an invalid GLE.
bool response(int ns, const double* a, const double* c, double dt, int obs, const double* lam,
              int64_t n, double* g, double* tau) {
    fth_gle gle;
    make_gle_struct(ns, a, c, &gle);
    double T[kMaxNs * kMaxNs], S[kMaxNs * kMaxNs];
    if (fth_gle_propagator(&gle, dt, T, S) != FTH_OK) return false;
    const int d = ns + 1;
    double G[kMaxD * kMaxD], Qn[kMaxD * kMaxD];
    const int x = obs == FTH_OBS_Q ? 0 : 1;
    for (int64_t i = 0; i < n; ++i) {
        mode_chain(ns, T, S, dt, lam[i], G, Qn);
        if (!mode_moments(d, G, Qn, x, &g[i], tau ? &tau[i] : nullptr)) return false;
    }
    return true;
}

// ------------------------------------------------------------------ target functions
bool target(int kind, const double* p, double x, double* f) {
    switch (kind) {
        case FTH_F_INV_SQRT: *f = 1.0 / std::sqrt(x); return x > 0.0;
        case FTH_F_FERMI: *f = 0.5 * (1.0 - std::tanh(0.5 * p[0] * (x - p[1]))); return true;
        case FTH_F_LOG: *f = std::log(x); return x > 1.0;          // must stay positive
        case FTH_F_EXP: *f = std::exp(-p[0] * x); return true;
        case FTH_F_POWER: *f = std::pow(x, p[0]); return x > 0.0;
        default: return false;
    }
}

// ------------------------------------------------------------------ the fit problem
struct Problem {
    int ns = 5, obs = 0, objective = 0;
    double dt = 0, delta = 1e-3, w_tau = 0, tau_ref = 0;
    std::vector<double> lam, f, logf;
    std::vector<char> tail;     // f < delta max f: upper bound only
    double fmax = 0, logcap = 0;
    int nparams() const { return ns * (ns + 1) / 2 + ns * (ns - 1) / 2 + ns * (ns + 1) / 2; }
    int nres() const { return (int)lam.size() + 1; }
};

// theta -> (A_p, B_p B_p^T)
void unpack(const Problem& P, const double* th, double* A, double* D) {
    const int ns = P.ns;
    double L[kMaxNs * kMaxNs] = {}, W[kMaxNs * kMaxNs] = {}, B[kMaxNs * kMaxNs] = {};
    int k = 0;
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j <= i; ++j, ++k) L[i * ns + j] = i == j ? std::exp(th[k]) : th[k];
    for (int i = 0; i < ns; ++i)
        for (int j = i + 1; j < ns; ++j, ++k) {
            W[i * ns + j] = th[k];
            W[j * ns + i] = -th[k];
        }
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j <= i; ++j, ++k) B[i * ns + j] = th[k];
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) {
            double s = 0.0, t = 0.0;
            for (int q = 0; q < ns; ++q) {
                s += L[i * ns + q] * L[j * ns + q];
                t += B[i * ns + q] * B[j * ns + q];
            }
            A[i * ns + j] = s + W[i * ns + j];
            D[i * ns + j] = t;
        }
}

// Drift, unscaled C_p, the response on the grid and the profiled scale gamma.
struct Eval {
    double A[kMaxNs * kMaxNs], C[kMaxNs * kMaxNs];
    std::vector<double> g, tau;
    double gamma = 1.0;
    bool ok = false;
};

bool evaluate(const Problem& P, const double* th, Eval& E, bool want_tau) {
    double D[kMaxNs * kMaxNs];
    unpack(P, th, E.A, D);
    E.ok = false;
    if (!lyap_continuous(P.ns, E.A, D, E.C)) return false;
    const int64_t n = (int64_t)P.lam.size();
    E.g.resize(n);
    E.tau.resize(n);
    if (!response(P.ns, E.A, E.C, P.dt, P.obs, P.lam.data(), n, E.g.data(),
                  want_tau ? E.tau.data() : nullptr))
        return false;
    if (P.objective == 0) {
        double s = 0.0;
        int cnt = 0;
        for (int64_t i = 0; i < n; ++i)
            if (!P.tail[i]) {
                s += P.logf[i] - std::log(E.g[i]);
                ++cnt;
            }
        E.gamma = cnt ? std::exp(s / cnt) : 1.0;
    } else {
        double fg = 0.0, gg = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            fg += P.f[i] * E.g[i];
            gg += E.g[i] * E.g[i];
        }
        E.gamma = gg > 0.0 ? fg / gg : 1.0;
    }
    E.ok = std::isfinite(E.gamma) && E.gamma > 0.0;
    return E.ok;
}

void residuals(const Problem& P, const double* th, double* r) {
    const int nr = P.nres();
    Eval E;
    const bool want_tau = P.w_tau > 0.0;
    if (!evaluate(P, th, E, want_tau)) {
        for (int i = 0; i < nr; ++i) r[i] = kBad;
        return;
    }
    const int64_t n = (int64_t)P.lam.size();
    const double lg = std::log(E.gamma);
    for (int64_t i = 0; i < n; ++i) {
        if (P.objective == 0) {
            const double v = std::log(E.g[i]) + lg;
            r[i] = P.tail[i] ? std::max(0.0, v - P.logcap) : v - P.logf[i];
        } else {
            r[i] = (E.gamma * E.g[i] - P.f[i]) / P.fmax;
        }
    }
    double pen = 0.0;
    if (want_tau) {
        double tmax = 0.0;
        for (int64_t i = 0; i < n; ++i) tmax = std::max(tmax, E.tau[i]);
        pen = P.w_tau * std::log(std::max(1.0, tmax / P.tau_ref));
    }
    r[n] = pen;
}

double cost_of(const std::vector<double>& r) {
    double s = 0.0;
    for (double x : r) s += x * x;
    return 0.5 * s;
}

// Seeded numbers for the starts (splitmix64; Box-Muller for normals).
struct Rng {
    uint64_t s;
    explicit Rng(uint64_t seed) : s(seed) {}
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double uniform(double a, double b) { return a + (b - a) * uniform(); }
    double normal() {
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

// Delta-like start: p coupled to damped oscillators (pairs of auxiliary momenta rotating
// at frequencies spread over [wmin, wmax]) plus, for an odd count, one fast friction term.
std::vector<double> initial(const Problem& P, double wmin, double wmax, Rng& g) {
    const int ns = P.ns;
    double a[kMaxNs * kMaxNs] = {};
    a[0] = wmin * std::exp(g.uniform(-1.0, 1.0));
    const int nosc = (ns - 1) / 2;
    const int nw = std::max(nosc, 1);
    double ws[kMaxNs];
    for (int k = 0; k < nw; ++k) {
        const double t = nw > 1 ? (double)k / (nw - 1) : 0.0;
        ws[k] = std::exp(std::log(wmin) + t * (std::log(wmax) - std::log(wmin)) + 0.3 * g.normal());
    }
    for (int k = 0; k < nosc; ++k) {
        const int i = 1 + 2 * k, j = 2 + 2 * k;
        const double w = ws[k];
        const double gam = w * std::exp(g.uniform(-2.5, -0.5));
        a[i * ns + i] = a[j * ns + j] = gam;
        a[i * ns + j] = w;
        a[j * ns + i] = -w;
        const double c = std::sqrt(gam * w) * std::exp(0.5 * g.normal());
        a[0 * ns + i] = c;
        a[i * ns + 0] = -c;
    }
    if ((ns - 1) % 2 == 1) {
        const int l = ns - 1;
        a[l * ns + l] = wmax * std::exp(g.uniform(-1.0, 0.0));
        const double c = std::sqrt(a[l * ns + l] * wmin);
        a[l] = c;
        a[l * ns] = -c;
    }
    // the symmetric part of this drift is diagonal and positive: L = its square root
    std::vector<double> th;
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j <= i; ++j)
            th.push_back(i == j ? 0.5 * std::log(a[i * ns + i] + 1e-3 * wmin) : 0.0);
    for (int i = 0; i < ns; ++i)
        for (int j = i + 1; j < ns; ++j) th.push_back(0.5 * (a[i * ns + j] - a[j * ns + i]));
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j <= i; ++j)
            th.push_back(i == j ? std::sqrt(a[i * ns + i] + 0.1 * wmin) * std::exp(0.3 * g.normal())
                                : 0.0);
    return th;
}

// Levenberg-Marquardt from th (in place); returns the final cost.
double levenberg_marquardt(const Problem& P, std::vector<double>& th, int max_iter,
                           int64_t* evals) {
    const int np = P.nparams(), nr = P.nres();
    std::vector<double> r(nr), rt(nr), J((size_t)nr * np), A((size_t)np * np), Ac((size_t)np * np);
    std::vector<double> grad(np), step(np), tt(np);
    residuals(P, th.data(), r.data());
    ++*evals;
    double cost = cost_of(r);
    double mu = 1e-3;
    int stall = 0;
    for (int it = 0; it < max_iter; ++it) {
        for (int j = 0; j < np; ++j) {
            const double h = 1e-7 * std::max(1.0, std::fabs(th[j]));
            tt = th;
            tt[j] += h;
            residuals(P, tt.data(), rt.data());
            ++*evals;
            for (int i = 0; i < nr; ++i) J[(size_t)i * np + j] = (rt[i] - r[i]) / h;
        }
        for (int a = 0; a < np; ++a) {
            double gs = 0.0;
            for (int i = 0; i < nr; ++i) gs += J[(size_t)i * np + a] * r[i];
            grad[a] = gs;
            for (int b = 0; b <= a; ++b) {
                double s = 0.0;
                for (int i = 0; i < nr; ++i) s += J[(size_t)i * np + a] * J[(size_t)i * np + b];
                A[(size_t)a * np + b] = A[(size_t)b * np + a] = s;
            }
        }
        bool accepted = false;
        while (mu < 1e12) {
            Ac = A;
            for (int a = 0; a < np; ++a) Ac[(size_t)a * np + a] += mu * (A[(size_t)a * np + a] + 1e-12);
            if (!cholesky(np, Ac.data())) {
                mu *= 10.0;
                continue;
            }
            for (int a = 0; a < np; ++a) step[a] = -grad[a];
            chol_solve(np, Ac.data(), step.data());
            for (int a = 0; a < np; ++a) tt[a] = th[a] + step[a];
            residuals(P, tt.data(), rt.data());
            ++*evals;
            const double c2 = cost_of(rt);
            if (c2 < cost) {
                const double gain = (cost - c2) / std::max(cost, 1e-300);
                th = tt;
                r = rt;
                cost = c2;
                mu = std::max(mu / 3.0, 1e-12);
                accepted = true;
                stall = gain < 1e-10 ? stall + 1 : 0;
                break;
            }
            mu *= 4.0;
        }
        if (!accepted || stall >= 5 || cost < 1e-28) break;
    }
    return cost;
}

}  // namespace

extern "C" {

fth_status fth_gle_response(const fth_gle* gle, double dt, int observable, const double* lambda,
                            int64_t n, double* g, double* tau) {
    if (!gle || !(dt > 0.0) || n < 0 || (n > 0 && (!lambda || !g)) || gle->s < 0 || gle->s > 4 ||
        (observable != FTH_OBS_P && observable != FTH_OBS_Q))
        return FTH_E_INVALID_ARG;
    // velocity Verlet is stable for lambda dt^2 < 4 only: beyond, no stationary state
    for (int64_t i = 0; i < n; ++i)
        if (!(lambda[i] > 0.0) || !(lambda[i] * dt * dt < 4.0)) return FTH_E_INVALID_ARG;
    const int ns = gle->s + 1;
    double a[kMaxNs * kMaxNs], c[kMaxNs * kMaxNs];
    for (int k = 0; k < ns * ns; ++k) {
        a[k] = gle->a_p[k];
        c[k] = gle->c_p[k];
    }
    return response(ns, a, c, dt, observable, lambda, n, g, tau) ? FTH_OK : FTH_E_INVALID_ARG;
}

fth_status fth_fit_gle(int f_kind, const double* f_params, double lambda_min, double lambda_max,
                       int s, double dt, const fth_fit_options* opt, fth_gle* out,
                       fth_fit_report* report) {
    fth_fit_options o{};
    o.w_tau = 0.2;                      // NULL options: the defaults documented in fth.h
    if (opt) o = *opt;
    if (!out || s < 1 || s > 4 || !(dt > 0.0) || !(lambda_min > 0.0) ||
        !(lambda_max > lambda_min) || !(lambda_max * dt * dt < 4.0) || o.npts < 0 || o.starts < 0 ||
        o.max_iter < 0 || o.delta < 0.0 || !(o.w_tau >= 0.0) || !std::isfinite(o.w_tau) ||
        (o.observable != FTH_OBS_P && o.observable != FTH_OBS_Q) ||
        (o.objective != FTH_FIT_AUTO && o.objective != FTH_FIT_LOG && o.objective != FTH_FIT_ABS))
        return FTH_E_INVALID_ARG;
    if ((f_kind == FTH_F_FERMI || f_kind == FTH_F_EXP || f_kind == FTH_F_POWER) && !f_params)
        return FTH_E_INVALID_ARG;
    Problem P;
    P.ns = s + 1;
    P.obs = o.observable;
    P.dt = dt;
    P.delta = o.delta > 0.0 ? o.delta : 1e-3;
    P.w_tau = o.w_tau;
    // internal objective: 0 log residuals (relative error), 1 absolute residuals / max f
    P.objective = o.objective == FTH_FIT_LOG ? 0
                : o.objective == FTH_FIT_ABS ? 1
                : (f_kind == FTH_F_FERMI ? 1 : 0);
    const int npts = o.npts > 0 ? o.npts : 120;
    const double l0 = std::log(lambda_min), l1 = std::log(lambda_max);
    for (int i = 0; i < npts; ++i) {
        const double lam = std::exp(npts > 1 ? l0 + (l1 - l0) * i / (npts - 1) : l0);
        double fv;
        if (!target(f_kind, f_params, lam, &fv) || !std::isfinite(fv) || !(fv >= 0.0))
            return FTH_E_INVALID_ARG;
        P.lam.push_back(lam);
        P.f.push_back(fv);
        P.fmax = std::max(P.fmax, fv);
    }
    if (!(P.fmax > 0.0)) return FTH_E_INVALID_ARG;
    for (int i = 0; i < npts; ++i) {
        P.tail.push_back(P.f[i] < P.delta * P.fmax ? 1 : 0);
        P.logf.push_back(std::log(std::max(P.f[i], 1e-300)));
    }
    P.logcap = std::log(P.delta * P.fmax);
    const double wmin = std::sqrt(lambda_min), wmax = std::sqrt(lambda_max);
    // correlation time of p^2 above which the penalty starts: that of a mode damped at
    // 0.2 of the lowest frequency, in samples
    P.tau_ref = 2.5 / (wmin * dt);

    const int starts = o.starts > 0 ? o.starts : 6;
    const int max_iter = o.max_iter > 0 ? o.max_iter : 400;
    std::vector<std::vector<double>> sol(starts);
    std::vector<double> costs(starts, std::numeric_limits<double>::infinity());
    std::atomic<int> next{0};
    std::atomic<int64_t> evals{0};
    auto worker = [&]() {
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= starts) return;
            Rng g(o.seed * 0x9E3779B97F4A7C15ull + 0x1234567ull * (uint64_t)(k + 1));
            std::vector<double> th = initial(P, wmin, wmax, g);
            int64_t ev = 0;
            costs[k] = levenberg_marquardt(P, th, max_iter, &ev);
            sol[k] = th;
            evals += ev;
        }
    };
    int nth = o.threads > 0 ? o.threads : (int)std::thread::hardware_concurrency();
    nth = std::max(1, std::min(nth, starts));
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    int best = -1;
    for (int k = 0; k < starts; ++k)
        if (std::isfinite(costs[k]) && (best < 0 || costs[k] < costs[best])) best = k;
    if (best < 0) return FTH_E_UNSUPPORTED;
    Eval E;
    if (!evaluate(P, sol[best].data(), E, true) || costs[best] >= 0.5 * kBad * kBad)
        return FTH_E_UNSUPPORTED;
    double cs[kMaxNs * kMaxNs];
    for (int k = 0; k < P.ns * P.ns; ++k) cs[k] = E.gamma * E.C[k];
    make_gle_struct(P.ns, E.A, cs, out);
    if (report) {
        std::memset(report, 0, sizeof *report);
        double mx = 0.0, ss = 0.0, mabs = 0.0, tail = 0.0, tmax = 0.0, ltmax = P.lam[0];
        int cnt = 0;
        for (int i = 0; i < npts; ++i) {
            const double gi = E.gamma * E.g[i];
            mabs = std::max(mabs, std::fabs(gi - P.f[i]) / P.fmax);
            if (P.tail[i]) {
                tail = std::max(tail, gi / P.fmax);
            } else {
                const double rel = std::fabs(gi / P.f[i] - 1.0);
                mx = std::max(mx, rel);
                ss += rel * rel;
                ++cnt;
            }
            if (E.tau[i] > tmax) {
                tmax = E.tau[i];
                ltmax = P.lam[i];
            }
        }
        report->max_rel_err = mx;
        report->rms_rel_err = cnt ? std::sqrt(ss / cnt) : 0.0;
        report->max_abs_err = mabs;
        report->tail_max = tail;
        report->tau_max = tmax;
        report->lambda_tau_max = ltmax;
        report->cost = costs[best];
        report->evaluations = evals.load();
        report->grid = npts;
        report->objective = P.objective == 0 ? FTH_FIT_LOG : FTH_FIT_ABS;
    }
    return FTH_OK;
}

}  // extern "C"
