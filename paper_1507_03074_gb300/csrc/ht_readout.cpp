// Track read-out of the peaks (host, FP64): Sec. 2 reads each peak's circle
// centre (A, B) as the radius rho = sqrt(A^2 + B^2) and the azimuth
// varphi = tan^-1(B / A) of the track (Fig. 1 compares both with a chi^2
// fit).  The transverse momentum of a unit charge follows from rho in the
// solenoid field: p_T [GeV] = 0.3 B [T] rho [m].
#include "ht_geom.h"

#include <cmath>
#include <string>

namespace hte {
ht_status report(ht_status s, const std::string &msg);
} // namespace hte

extern "C" ht_status ht_track_params(const ht_binning *binning, const ht_ranges *ranges, const ht_peak *peaks,
                                     uint32_t n, double b_field_t, ht_track *out)
{
    std::string why;
    if (!binning || !ranges || (n && (!peaks || !out)))
        return hte::report(HT_E_INVAL, "NULL argument");
    if (!htg::validate(binning, ranges, 1, &why))
        return hte::report(HT_E_INVAL, why);
    if (!(std::isfinite(b_field_t) && b_field_t > 0.0))
        return hte::report(HT_E_INVAL, "b_field_t must be finite and > 0");
    for (uint32_t k = 0; k < n; ++k) {
        const ht_peak &p = peaks[k];
        if (p.itheta >= binning->n_theta || p.iphi >= binning->n_phi || p.ia >= binning->n_a ||
            p.ib >= binning->n_b)
            return hte::report(HT_E_INVAL, "peak " + std::to_string(k) + " lies outside the binning");
    }
    const double a0 = ranges->a_min, da = ((double)ranges->a_max - a0) / binning->n_a;
    const double b0 = ranges->b_min, db = ((double)ranges->b_max - b0) / binning->n_b;
    const double t0 = htg::snap_quarter(ranges->theta_min);
    const double dt = (htg::snap_quarter(ranges->theta_max) - t0) / binning->n_theta;
    const double f0 = htg::snap_quarter(ranges->phi_min);
    const double df = (htg::snap_quarter(ranges->phi_max) - f0) / binning->n_phi;
    for (uint32_t k = 0; k < n; ++k) {
        const ht_peak &p = peaks[k];
        ht_track &t = out[k];
        t.a = a0 + (p.ia + 0.5) * da;
        t.b = b0 + (p.ib + 0.5) * db;
        t.rho = std::hypot(t.a, t.b);
        t.varphi = std::atan2(t.b, t.a);
        t.pt = 0.3 * b_field_t * t.rho / 1000.0;
        t.theta = t0 + (p.itheta + 0.5) * dt;
        t.eta = -std::log(std::tan(0.5 * t.theta));
        t.phi_c = f0 + (p.iphi + 0.5) * df;
        t.votes = p.votes;
        t.event = p.event;
    }
    return HT_OK;
}
