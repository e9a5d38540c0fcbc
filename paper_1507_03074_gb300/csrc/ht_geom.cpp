// Host-side geometry of the Hough space: argument validation and the FP32
// pseudo-angle edge tables the kernels bin hits with.
//
// Binning of the angles (Sec. 2 lists theta and phi among the four binned
// Hough dimensions): uniform bins in the polar angle theta (from +z) and the
// azimuth phi.  To make the bin of a hit bit-reproducible without atan2, the
// kernels compare a monotone pseudo-angle of the hit (built from + - / sqrt
// only) with the pseudo-angle of each uniform edge, computed here once in
// double precision and rounded to float.  Multiples of pi/4 take their exact
// pseudo-angles (theta = m pi/4 -> m/2, phi = m pi/4 -> (m + 4)/2).
#include "ht_geom.h"

#include <cmath>
#include <cstdio>
#include <cstring>

namespace htg {

static const double kPi = 3.14159265358979323846;
static const double kQuarter = kPi / 4.0;

double snap_quarter(double a)
{
    const double q = a / kQuarter;
    const double m = std::nearbyint(q);
    return std::fabs(q - m) < 1e-6 ? m * kQuarter : a;
}

static bool exact_quarter(double a, long *m)
{
    const double q = a / kQuarter;
    const double r = std::nearbyint(q);
    if (std::fabs(q - r) < 1e-9) {
        *m = (long)r;
        return true;
    }
    return false;
}

// Pseudo-angle of the polar angle th in [0, pi]: rho/(z + rho) for z >= 0,
// else 1 + (-z)/(rho - z), with (rho, z) = (sin th, cos th).
static double theta_pseudo64(double th)
{
    const double z = std::cos(th), rho = std::sin(th);
    return z >= 0.0 ? rho / (z + rho) : 1.0 + (-z) / (rho - z);
}

// Pseudo-angle of the azimuth ph: the quadrant diamond angle of
// (u, v) = (-cos ph, -sin ph), which is 0 at ph = -pi and 4 at ph = +pi.
static double phi_pseudo64(double ph)
{
    const double u = -std::cos(ph), v = -std::sin(ph);
    if (v >= 0.0)
        return u >= 0.0 ? v / (u + v) : 1.0 + (-u) / ((-u) + v);
    return u < 0.0 ? 2.0 + (-v) / ((-u) + (-v)) : 3.0 + u / (u + (-v));
}

void theta_edges(float lo, float hi, uint32_t n, float *e)
{
    const double a = snap_quarter(lo), b = snap_quarter(hi);
    for (uint32_t k = 0; k <= n; ++k) {
        const double th = a + (double)k * (b - a) / (double)n;
        long m;
        e[k] = (float)(exact_quarter(th, &m) ? 0.5 * (double)m : theta_pseudo64(th));
    }
}

void phi_edges(float lo, float hi, uint32_t n, float *e)
{
    const double a = snap_quarter(lo), b = snap_quarter(hi);
    for (uint32_t k = 0; k <= n; ++k) {
        const double ph = a + (double)k * (b - a) / (double)n;
        long m;
        e[k] = (float)(exact_quarter(ph, &m) ? 0.5 * (double)(m + 4) : phi_pseudo64(ph));
    }
}

// Bin width fl((hi - lo) / n) in FP32.
float delta(float lo, float hi, uint32_t n)
{
    volatile float w = hi - lo, fn = (float)n;
    volatile float d = w / fn;
    return d;
}

// The B bin of the vote, floor(fl(fl(B - b_min) / dB)) for 0 <= t < n_b, is a
// non-decreasing step function of the float B (each FP32 step is a rounded
// monotone operation).  beta[k] is the smallest float B whose bin is >= k
// (k = 0 .. n_b; bin = -1 below range, n_b above), so for any float B:
//   in range  <=>  beta[0] <= B < beta[n_b],   bin = max{k : beta[k] <= B}.
// Each threshold is found by a binary search over the floats (in their
// integer order) between two bracketing values, evaluating the same FP32
// operations as the vote.
static int b_bin_f32(float B, float b_min, float db, uint32_t nb)
{
    volatile float num = B - b_min;
    volatile float t = num / db;
    if (!(t >= 0.0f))
        return -1;
    if (!(t < (float)nb))
        return (int)nb;
    return (int)(uint32_t)t;
}

// Floats in increasing order <-> integers in increasing order (+0 and -0 share 0).
static int64_t float_key(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (u & 0x80000000u) ? -(int64_t)(u & 0x7fffffffu) : (int64_t)u;
}

static float key_float(int64_t k)
{
    const uint32_t u = k >= 0 ? (uint32_t)k : (0x80000000u | (uint32_t)(-k));
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

void b_thresholds(float b_min, float db, uint32_t nb, float *beta)
{
    for (uint32_t k = 0; k <= nb; ++k) {
        // bracket: lo two bins below (bin < k), hi two bins above (bin >= k)
        float lo = (float)((double)b_min + ((double)k - 2.0) * (double)db);
        float hi = (float)((double)b_min + ((double)k + 2.0) * (double)db);
        for (int widen = 0; b_bin_f32(lo, b_min, db, nb) >= (int)k && widen < 64; ++widen)
            lo = lo - std::fabs(lo) - db;
        for (int widen = 0; b_bin_f32(hi, b_min, db, nb) < (int)k && widen < 64; ++widen)
            hi = hi + std::fabs(hi) + db;
        // smallest float key in (key(lo), key(hi)] whose bin is >= k
        int64_t a = float_key(lo), c = float_key(hi);
        while (c - a > 1) {
            const int64_t m = a + (c - a) / 2;
            if (b_bin_f32(key_float(m), b_min, db, nb) >= (int)k)
                c = m;
            else
                a = m;
        }
        beta[k] = key_float(c);
    }
}

bool phi_is_full_circle(float lo, float hi)
{
    return snap_quarter(lo) == -kPi && snap_quarter(hi) == kPi;
}

uint32_t max_admit(const ht_binning &b)
{
    uint64_t t = 2ull * b.win_theta + 1, p = 2ull * b.win_phi + 1;
    if (t > b.n_theta) t = b.n_theta;
    if (p > b.n_phi) p = b.n_phi;
    return (uint32_t)(t * p);
}

static bool finite_all(const ht_ranges &r)
{
    const float v[8] = {r.theta_min, r.theta_max, r.phi_min, r.phi_max, r.a_min, r.a_max, r.b_min, r.b_max};
    for (float f : v)
        if (!std::isfinite(f))
            return false;
    return true;
}

bool validate(const ht_binning *b, const ht_ranges *r, uint32_t threshold, std::string *why)
{
    char buf[256];
    if (!b || !r) {
        *why = "binning and ranges must not be NULL";
        return false;
    }
    if (b->n_theta < 1 || b->n_theta > 1024 || b->n_phi < 1 || b->n_phi > 1024 ||
        (uint64_t)b->n_theta * b->n_phi > 8192) {
        *why = "need 1 <= n_theta, n_phi <= 1024 and n_theta*n_phi <= 8192";
        return false;
    }
    if (b->n_a < 1 || b->n_a > 65535 || b->n_b < 1 || b->n_b > 65535) {
        *why = "need 1 <= n_a, n_b <= 65535";
        return false;
    }
    const uint64_t cells = (uint64_t)b->n_theta * b->n_phi * b->n_a * b->n_b;
    if (cells >= (1ull << 32)) {
        std::snprintf(buf, sizeof buf, "matrix of %llu cells: need fewer than 2^32",
                      (unsigned long long)cells);
        *why = buf;
        return false;
    }
    if (threshold < 1) {
        *why = "threshold must be >= 1";
        return false;
    }
    if (!finite_all(*r) || !(r->theta_min < r->theta_max) || !(r->phi_min < r->phi_max) ||
        !(r->a_min < r->a_max) || !(r->b_min < r->b_max)) {
        *why = "ranges must be finite with min < max";
        return false;
    }
    const double t0 = snap_quarter(r->theta_min), t1 = snap_quarter(r->theta_max);
    const double p0 = snap_quarter(r->phi_min), p1 = snap_quarter(r->phi_max);
    if (t0 < 0.0 || t1 > kPi || p0 < -kPi || p1 > kPi) {
        *why = "need 0 <= theta_min < theta_max <= pi and -pi <= phi_min < phi_max <= pi";
        return false;
    }
    return true;
}

} // namespace htg
