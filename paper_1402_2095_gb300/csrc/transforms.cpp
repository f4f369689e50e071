// Spectral scaling and shift, GLE rescaling and the inverse transforms (host, FP64):
// fth_spectral_map, fth_gle_scale, fth_untransform, fth_untransform_trace.
//
// Sec. "The f-thermostat" reuses one fitted GLE for other spectra: with A_p -> alpha A_p
// and C_p -> gamma C_p the sampled <p p^T> becomes gamma f((r M + m I) / alpha^2) for a
// GLE fitted to f and the input r M + m I.  The paper's benchmarks then map the sampled
// quantity back to the wanted one: ln M = ln(r M) - I ln r (a logarithm fitted on a range
// the scaled spectrum falls into), exp(-a M) = exp(-a (M + m I)) e^{a m} (a shift that
// makes an indefinite M positive definite), and for a power law f(x) = x^k,
// f(M) = f(r M) r^{-k}.  The printed shift has its sign flipped; the map here solves
// r lo + m = lo' and r hi + m = hi' directly.
#include <cmath>
#include <cstring>

#include "fth.h"

extern "C" {

fth_status fth_spectral_map(double lo, double hi, double lo_target, double hi_target, double* r,
                            double* m) {
    if (!r || !m || !(hi > lo) || !(hi_target > lo_target) || !std::isfinite(lo) ||
        !std::isfinite(hi) || !std::isfinite(lo_target) || !std::isfinite(hi_target))
        return FTH_E_INVALID_ARG;
    *r = (hi_target - lo_target) / (hi - lo);
    *m = (lo_target * hi - hi_target * lo) / (hi - lo);
    return FTH_OK;
}

fth_status fth_gle_scale(const fth_gle* in, double alpha, double gamma, fth_gle* out) {
    if (!in || !out || in->s < 0 || in->s > 4 || !(alpha > 0.0) || !(gamma > 0.0) ||
        !std::isfinite(alpha) || !std::isfinite(gamma))
        return FTH_E_INVALID_ARG;
    fth_gle g;
    std::memcpy(&g, in, sizeof g);
    const int ns = in->s + 1;
    for (int k = 0; k < ns * ns; ++k) {
        g.a_p[k] = alpha * in->a_p[k];
        g.c_p[k] = gamma * in->c_p[k];
    }
    std::memcpy(out, &g, sizeof g);
    return FTH_OK;
}

static bool untransform_params(int kind, const double* p) {
    if (!p) return false;
    switch (kind) {
        case FTH_U_LOG_SCALED: return p[0] > 0.0 && std::isfinite(p[0]);
        case FTH_U_EXP_SHIFTED: return std::isfinite(p[0]) && std::isfinite(p[1]);
        case FTH_U_POWER_SCALED: return p[0] > 0.0 && std::isfinite(p[0]) && std::isfinite(p[1]);
        default: return false;
    }
}

fth_status fth_untransform(int kind, const double* params, const int64_t* pairs, int64_t k,
                           double* values, double* errbars) {
    if (!untransform_params(kind, params) || k < 0 || (k > 0 && (!values || !pairs)))
        return FTH_E_INVALID_ARG;
    for (int64_t e = 0; e < k; ++e) {
        switch (kind) {
            case FTH_U_LOG_SCALED:      // ln M = ln(r M) - I ln r: the diagonal only
                if (pairs[2 * e] == pairs[2 * e + 1]) values[e] -= std::log(params[0]);
                break;
            case FTH_U_EXP_SHIFTED: {   // exp(-a M) = exp(-a (M + m I)) e^{a m}
                const double s = std::exp(params[0] * params[1]);
                values[e] *= s;
                if (errbars) errbars[e] *= s;
                break;
            }
            default: {                  // f(M) = f(r M) r^-k for f(x) = x^k
                const double s = std::pow(params[0], -params[1]);
                values[e] *= s;
                if (errbars) errbars[e] *= s;
            }
        }
    }
    return FTH_OK;
}

fth_status fth_untransform_trace(int kind, const double* params, int64_t n, double* value,
                                 double* errbar) {
    if (!untransform_params(kind, params) || n < 1 || !value) return FTH_E_INVALID_ARG;
    switch (kind) {
        case FTH_U_LOG_SCALED: *value -= (double)n * std::log(params[0]); break;
        case FTH_U_EXP_SHIFTED: {
            const double s = std::exp(params[0] * params[1]);
            *value *= s;
            if (errbar) *errbar *= s;
            break;
        }
        default: {
            const double s = std::pow(params[0], -params[1]);
            *value *= s;
            if (errbar) *errbar *= s;
        }
    }
    return FTH_OK;
}

}  // extern "C"
