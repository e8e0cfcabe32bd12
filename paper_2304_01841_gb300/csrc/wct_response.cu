// Field-response ingestion: the tick-sampled detector response of §2 step 3 ("convolved with
// the detector response") built from a field response (currents induced on one wire for drift
// paths across the pitch, on a fine time grid) and an electronics impulse response.  Host
// code in FP64, run once per configuration; the result feeds wct_sim_create (folded mode) or
// wct_sim_set_impact_responses (impact mode).
//
// For impact phase p (charge at y_p = ((p + 1/2) / n_imp - 1/2) pitch from its wire's centre)
// and response row r (wire offset d = r - K), the charge sits at x = y_p - d pitch from the
// responding wire, so that wire's current is the field's I(x, t): linear interpolation
// between the two paths around x (|x| when the field is given on one side only), zero beyond
// the outermost path.  It is convolved in time with the electronics response on the fine
// grid and sampled every m = tick / period samples:
//     R_p[r][tau] = period * sum_s I(x, s) E[tau m - s].
#include "wct_sim.h"

#include <cmath>
#include <vector>

namespace {

bool finite_all(const double *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Linear interpolation of the path currents at position x (already mirrored); false when x
// lies outside [pos[0], pos[n - 1]].
bool interpolate(const wct_field_response_t &f, double x, std::vector<double> &out) {
    const int n = f.n_paths;
    if (x < f.path_pos_mm[0] || x > f.path_pos_mm[n - 1]) return false;
    int j = 0;
    while (j + 2 < n && f.path_pos_mm[j + 1] <= x) ++j;   // pos[j] <= x <= pos[j + 1]
    const double a = (x - f.path_pos_mm[j]) / (f.path_pos_mm[j + 1] - f.path_pos_mm[j]);
    const double *lo = f.current + (size_t)j * f.n_samples;
    const double *hi = lo + f.n_samples;
    for (int s = 0; s < f.n_samples; ++s) out[s] = (1.0 - a) * lo[s] + a * hi[s];
    return true;
}

}  // namespace

extern "C" wct_status_t wct_response_from_field(const wct_field_response_t *field, const double *electronics,
                                                int32_t n_elec, double pitch_mm, int32_t n_impact, double tick_us,
                                                int32_t n_wires_resp, int32_t n_ticks_resp, float *impact_out,
                                                float *folded_out) {
    if (!field || !electronics || n_elec < 1 || !field->path_pos_mm || !field->current) return WCT_EINVAL;
    const wct_field_response_t &f = *field;
    if (f.n_paths < 2 || f.n_samples < 1 || !(f.period_us > 0.0) || !std::isfinite(f.period_us)) return WCT_EINVAL;
    if (!(pitch_mm > 0.0) || !std::isfinite(pitch_mm) || n_impact < 1 || n_impact > 4096) return WCT_EINVAL;
    if (!(tick_us > 0.0) || !std::isfinite(tick_us)) return WCT_EINVAL;
    if (n_wires_resp < 1 || (n_wires_resp & 1) == 0 || n_wires_resp > WCT_MAX_RESPONSE_WIRES) return WCT_EINVAL;
    if (n_ticks_resp < 1 || n_ticks_resp > 65536) return WCT_EINVAL;
    const double ratio = tick_us / f.period_us;
    const long long m = std::llround(ratio);
    if (m < 1 || std::fabs(ratio - (double)m) > 1e-9 * ratio) return WCT_EINVAL;
    for (int j = 0; j + 1 < f.n_paths; ++j)
        if (!(f.path_pos_mm[j + 1] > f.path_pos_mm[j])) return WCT_EINVAL;
    if (!finite_all(f.path_pos_mm, (size_t)f.n_paths) ||
        !finite_all(f.current, (size_t)f.n_paths * (size_t)f.n_samples) || !finite_all(electronics, (size_t)n_elec))
        return WCT_EINVAL;
    const bool mirror = f.path_pos_mm[0] >= 0.0;
    const int K = n_wires_resp / 2;
    const size_t plane = (size_t)n_wires_resp * n_ticks_resp;
    std::vector<double> folded(plane, 0.0), cur(f.n_samples), row(n_ticks_resp);
    for (int p = 0; p < n_impact; ++p) {
        const double y = ((p + 0.5) / n_impact - 0.5) * pitch_mm;
        for (int r = 0; r < n_wires_resp; ++r) {
            double x = y - (double)(r - K) * pitch_mm;
            if (mirror) x = std::fabs(x);
            const bool any = interpolate(f, x, cur);
            for (int t = 0; t < n_ticks_resp; ++t) {
                double acc = 0.0;
                if (any) {
                    const long long n = (long long)t * m;   // fine-grid index of the tick time
                    const long long s_lo = n - (n_elec - 1) > 0 ? n - (n_elec - 1) : 0;
                    const long long s_hi = n < f.n_samples - 1 ? n : f.n_samples - 1;
                    for (long long s = s_lo; s <= s_hi; ++s) acc += cur[(size_t)s] * electronics[n - s];
                    acc *= f.period_us;
                }
                row[t] = acc;
            }
            const size_t off = (size_t)r * n_ticks_resp;
            if (impact_out)
                for (int t = 0; t < n_ticks_resp; ++t) impact_out[(size_t)p * plane + off + t] = (float)row[t];
            for (int t = 0; t < n_ticks_resp; ++t) folded[off + t] += row[t];
        }
    }
    if (folded_out)
        for (size_t i = 0; i < plane; ++i) folded_out[i] = (float)(folded[i] / n_impact);
    return WCT_OK;
}
