// Drives the library's host-only code -- argument validation, the angle
// edge tables, the B-bin thresholds and the track read-out -- over valid,
// degenerate and invalid inputs, for a build with AddressSanitizer and
// UndefinedBehaviorSanitizer (the CUDA parts are not built here).
#include <cmath>
#include <cstdio>
#include <limits>
#include <string>
#include <vector>

#include "ht_geom.h"

namespace hte {
ht_status report(ht_status s, const std::string &) { return s; }   // the library's error text goes to ht_last_error
} // namespace hte

extern "C" ht_status ht_track_params(const ht_binning *, const ht_ranges *, const ht_peak *, uint32_t, double,
                                     ht_track *);

int main()
{
    int bad = 0;
    const float pi = 3.14159274f, nan = std::numeric_limits<float>::quiet_NaN();
    const ht_ranges full{0.f, pi, -pi, pi, -2000.f, 2000.f, -2000.f, 2000.f};
    const ht_ranges part{0.4f, 2.6f, -2.0f, 1.5f, -1500.f, 1700.f, -900.f, 2100.f};
    const ht_binning bins[] = {{4, 16, 1024, 1024, 0, 0}, {3, 5, 37, 29, 1, 1}, {8, 32, 2048, 2048, 0, 0},
                               {1, 1, 1, 1, 0, 0}, {1024, 8, 2, 2, 0, 3}};
    for (const ht_binning &b : bins)
        for (const ht_ranges *r : {&full, &part}) {
            std::string why;
            if (!htg::validate(&b, r, 10, &why)) {
                bad |= 1;
                continue;
            }
            std::vector<float> et(b.n_theta + 1), ep(b.n_phi + 1), beta(b.n_b + 1);
            htg::theta_edges(r->theta_min, r->theta_max, b.n_theta, et.data());
            htg::phi_edges(r->phi_min, r->phi_max, b.n_phi, ep.data());
            htg::b_thresholds(r->b_min, htg::delta(r->b_min, r->b_max, b.n_b), b.n_b, beta.data());
            for (uint32_t k = 1; k <= b.n_b; ++k)
                bad |= !(beta[k - 1] < beta[k]);
            std::vector<ht_peak> pk(5);
            for (uint32_t k = 0; k < pk.size(); ++k)
                pk[k] = ht_peak{k % b.n_theta, k % b.n_phi, (k * 7) % b.n_a, (k * 13) % b.n_b, 10 + k, 0.f, 0.f, 0};
            std::vector<ht_track> tr(pk.size());
            bad |= ht_track_params(&b, r, pk.data(), (uint32_t)pk.size(), 2.0, tr.data()) != HT_OK;
            for (const ht_track &t : tr)
                bad |= !(std::isfinite(t.rho) && t.rho >= 0.0 && std::isfinite(t.varphi));
            pk[0].ia = b.n_a;   // outside the binning: refused
            bad |= ht_track_params(&b, r, pk.data(), (uint32_t)pk.size(), 2.0, tr.data()) != HT_E_INVAL;
        }
    // invalid arguments are refused, not read past
    std::string why;
    const ht_binning zero{0, 16, 1024, 1024, 0, 0}, huge{1024, 1024, 65535, 65535, 0, 0};
    const ht_ranges empty{1.f, 1.f, -pi, pi, -2000.f, 2000.f, -2000.f, 2000.f};
    const ht_ranges nanr{nan, pi, -pi, pi, -2000.f, 2000.f, -2000.f, 2000.f};
    bad |= htg::validate(&zero, &full, 10, &why);
    bad |= htg::validate(&huge, &full, 10, &why);
    bad |= htg::validate(&bins[0], &empty, 10, &why);
    bad |= htg::validate(&bins[0], &nanr, 10, &why);
    bad |= htg::validate(&bins[0], &full, 0, &why);
    bad |= htg::validate(nullptr, &full, 10, &why);
    bad |= ht_track_params(&bins[0], &full, nullptr, 3, 2.0, nullptr) != HT_E_INVAL;
    bad |= ht_track_params(&bins[0], &full, nullptr, 0, nan, nullptr) != HT_E_INVAL;
    std::printf(bad ? "FAIL\n" : "OK\n");
    return bad;
}
