/*
 * Hough-Transform track finder: plain, slow, scalar CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg use it.  It shares no code, header, table or
 * helper with the CUDA library; it is compiled on its own with
 *     gcc -O2 -ffp-contract=off -fno-fast-math
 * so that every float operation below is one IEEE-754 binary32 operation
 * rounded to nearest-even, exactly in the order written.
 *
 * What it computes (paper: "GPGPU for track finding in High Energy Physics",
 * Sec. 2 and Sec. 3):
 *   Step 1 (Sec. 2): every hit (x,y,z) votes for all circles through itself
 *   and the interaction point, x^2 + y^2 - 2Ax - 2By = 0, i.e. for every A
 *   bin the B = (x^2 + y^2 - 2Ax) / (2y); the cell M_H(theta,phi,A,B) is
 *   incremented by one.  Sec. 3 fixes the loop structure "for each A, the
 *   corresponding B is evaluated".
 *   Step 2 (Sec. 2, Sec. 3): cells above a threshold that are local maxima
 *   among their neighbours are the tracks.
 *
 * The paper leaves the following open; the readings taken here are:
 *   R1 axis sizes: (theta, phi, A, B) = 4 x 16 x 1024 x 1024 for the paper's
 *      binning (Sec. 2 lists the four sizes in a garbled order); the matrix is
 *      M[theta][phi][A][B], B fastest.
 *   R2 a hit enters the (theta, phi) slice that contains its own polar angle
 *      (from the +z beam axis) and azimuth, plus +-win_theta / +-win_phi
 *      neighbouring bins (phi wraps iff the phi range is the full circle).
 *   R3 the angle bins are found without transcendental functions: a
 *      "pseudo-angle" built from + - / sqrt is compared with FP32 edge tables
 *      that hold the same pseudo-angle of the uniform angle edges.
 *   R4 A is the bin centre; B is found by the division form; the B bin is
 *      floor((B - b_min) / dB) by IEEE division; out-of-range votes drop.
 *   R5 threshold means votes >= T.
 *   R6 the neighbours are the 8 cells of the (A,B) plane of the same slice.
 *   R7 ties: a cell is a peak iff it is > every neighbour with a smaller
 *      linear index and >= every neighbour with a larger linear index.
 *   R8 peaks are reported in ascending linear-index order.
 *   R9 the counters are uint32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HO_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Geometry: pseudo-angles (R3).                                             */
/* ------------------------------------------------------------------------ */

/* Snap an angle given as float to the nearest multiple of pi/4 if it lies
 * within float rounding of it (so that the float -pi, pi, pi/2 ... of a
 * caller mean the exact angles). */
static double ho_snap(double a)
{
    double q = a / (HO_PI / 4.0);
    double m = nearbyint(q);
    if (fabs(q - m) < 1e-6)
        return m * (HO_PI / 4.0);
    return a;
}

/* If the exact angle a (double) is a multiple m of pi/4, set *m and return 1. */
static int ho_quarter(double a, long *m)
{
    double q = a / (HO_PI / 4.0);
    double r = nearbyint(q);
    if (fabs(q - r) < 1e-9) {
        *m = (long)r;
        return 1;
    }
    return 0;
}

/* Polar pseudo-angle of the direction (rho, z), rho >= 0: 0 along +z, 1 in
 * the transverse plane, 2 along -z.  Monotone in the polar angle. */
static float ho_theta_pseudo_f32(float rho, float z)
{
    if (z >= 0.0f) {
        float den = z + rho;
        return rho / den;
    } else {
        float mz = -z;
        float den = rho - z;
        float q = mz / den;
        return 1.0f + q;
    }
}

/* Azimuthal pseudo-angle of (x, y) measured from the -pi direction, in
 * [0, 4]: the "diamond angle" of (u, v) = (-x, -y), one unit per quadrant. */
static float ho_phi_pseudo_f32(float x, float y)
{
    float u = -x, v = -y;
    if (v >= 0.0f) {
        if (u >= 0.0f) {
            float den = u + v;
            return v / den;
        } else {
            float mu = -u;
            float den = mu + v;
            float q = mu / den;
            return 1.0f + q;
        }
    } else {
        if (u < 0.0f) {
            float mu = -u, mv = -v;
            float den = mu + mv;
            float q = mv / den;
            return 2.0f + q;
        } else {
            float mv = -v;
            float den = u + mv;
            float q = u / den;
            return 3.0f + q;
        }
    }
}

/* The same two pseudo-angles, in double, of an exact angle. */
static double ho_theta_pseudo_f64(double th)
{
    double c = cos(th), s = sin(th);
    if (c >= 0.0)
        return s / (c + s);
    return 1.0 + (-c) / (s - c);
}

static double ho_phi_pseudo_f64(double ph)
{
    double u = -cos(ph), v = -sin(ph);
    if (v >= 0.0) {
        if (u >= 0.0)
            return v / (u + v);
        return 1.0 + (-u) / ((-u) + v);
    }
    if (u < 0.0)
        return 2.0 + (-v) / ((-u) + (-v));
    return 3.0 + u / (u + (-v));
}

/* Edge tables: e[k] = pseudo-angle of the k-th uniform angle edge, k=0..n,
 * evaluated in double and rounded once to float; multiples of pi/4 take
 * their exact pseudo-angles. */
static void ho_edges_theta(float tmin, float tmax, uint32_t n, float *e)
{
    double a = ho_snap((double)tmin), b = ho_snap((double)tmax);
    for (uint32_t k = 0; k <= n; ++k) {
        double th = a + (double)k * (b - a) / (double)n;
        long m;
        double d;
        if (ho_quarter(th, &m))
            d = 0.5 * (double)m;             /* theta = m*pi/4 -> m/2 */
        else
            d = ho_theta_pseudo_f64(th);
        e[k] = (float)d;
    }
}

static void ho_edges_phi(float pmin, float pmax, uint32_t n, float *e)
{
    double a = ho_snap((double)pmin), b = ho_snap((double)pmax);
    for (uint32_t k = 0; k <= n; ++k) {
        double ph = a + (double)k * (b - a) / (double)n;
        long m;
        double d;
        if (ho_quarter(ph, &m))
            d = 0.5 * (double)(m + 4);       /* phi = m*pi/4 -> (m+4)/2 */
        else
            d = ho_phi_pseudo_f64(ph);
        e[k] = (float)d;
    }
}

/* ------------------------------------------------------------------------ */
/* Parameters.  bins = {n_theta, n_phi, n_a, n_b, win_theta, win_phi};       */
/* rng = {theta_min, theta_max, phi_min, phi_max, a_min, a_max, b_min, b_max}*/
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t nt, np, na, nb, wt, wp;
    float a_min, b_min, da, db;
    int phi_full;
    float *et, *ep;
} ho_geom;

static int ho_geom_init(ho_geom *g, const uint32_t *bins, const float *rng)
{
    g->nt = bins[0]; g->np = bins[1]; g->na = bins[2]; g->nb = bins[3];
    g->wt = bins[4]; g->wp = bins[5];
    if (!g->nt || !g->np || !g->na || !g->nb)
        return -1;
    g->a_min = rng[4];
    g->b_min = rng[6];
    g->da = (rng[5] - rng[4]) / (float)g->na;     /* dA = fl((a_max-a_min)/N_A) */
    g->db = (rng[7] - rng[6]) / (float)g->nb;     /* dB = fl((b_max-b_min)/N_B) */
    g->phi_full = (ho_snap(rng[2]) == -HO_PI && ho_snap(rng[3]) == HO_PI);
    g->et = (float *)malloc(sizeof(float) * (g->nt + 1));
    g->ep = (float *)malloc(sizeof(float) * (g->np + 1));
    if (!g->et || !g->ep)
        return -2;
    ho_edges_theta(rng[0], rng[1], g->nt, g->et);
    ho_edges_phi(rng[2], rng[3], g->np, g->ep);
    return 0;
}

static void ho_geom_free(ho_geom *g)
{
    free(g->et);
    free(g->ep);
}

/* bin = #{k = 1..n-1 : D >= e[k]}; the caller has checked e[0] <= D <= e[n]. */
static uint32_t ho_bin_of(float D, const float *e, uint32_t n)
{
    uint32_t b = 0;
    for (uint32_t k = 1; k < n; ++k)
        if (D >= e[k])
            ++b;
    return b;
}

/* Slice admission of one hit (R2, R3).  Writes the admitted slices
 * s = itheta*n_phi + iphi into out (ascending itheta, then the phi window
 * from -win to +win) and returns their number; 0 drops the hit. */
static uint32_t ho_admit(const ho_geom *g, float x, float y, float z, uint32_t *out)
{
    float r2 = x * x + y * y;
    float rho = sqrtf(r2);
    if (!(rho > 0.0f))
        return 0;
    float dt = ho_theta_pseudo_f32(rho, z);
    float dp = ho_phi_pseudo_f32(x, y);
    if (!(dt >= g->et[0] && dt <= g->et[g->nt]))
        return 0;
    if (!(dp >= g->ep[0] && dp <= g->ep[g->np]))
        return 0;
    uint32_t it = ho_bin_of(dt, g->et, g->nt);
    uint32_t ip = ho_bin_of(dp, g->ep, g->np);
    long t0 = (long)it - (long)g->wt, t1 = (long)it + (long)g->wt;
    if (t0 < 0) t0 = 0;
    if (t1 > (long)g->nt - 1) t1 = (long)g->nt - 1;
    uint32_t cnt = 0;
    for (long t = t0; t <= t1; ++t) {
        if (g->phi_full) {
            if (2 * (long)g->wp + 1 >= (long)g->np) {
                for (uint32_t p = 0; p < g->np; ++p)
                    out[cnt++] = (uint32_t)t * g->np + p;
            } else {
                for (long d = -(long)g->wp; d <= (long)g->wp; ++d) {
                    long p = ((long)ip + d) % (long)g->np;
                    if (p < 0) p += g->np;
                    out[cnt++] = (uint32_t)t * g->np + (uint32_t)p;
                }
            }
        } else {
            long p0 = (long)ip - (long)g->wp, p1 = (long)ip + (long)g->wp;
            if (p0 < 0) p0 = 0;
            if (p1 > (long)g->np - 1) p1 = (long)g->np - 1;
            for (long p = p0; p <= p1; ++p)
                out[cnt++] = (uint32_t)t * g->np + (uint32_t)p;
        }
    }
    return cnt;
}

static uint32_t ho_max_admit(const ho_geom *g)
{
    uint32_t nt = 2 * g->wt + 1, np = 2 * g->wp + 1;
    if (nt > g->nt) nt = g->nt;
    if (np > g->np) np = g->np;
    return nt * np;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points.                                                    */
/* ------------------------------------------------------------------------ */

/* theta_edges[n_theta+1], phi_edges[n_phi+1]. */
int ho_edges(const uint32_t *bins, const float *rng, float *theta_edges, float *phi_edges)
{
    ho_geom g;
    if (ho_geom_init(&g, bins, rng))
        return -1;
    memcpy(theta_edges, g.et, sizeof(float) * (g.nt + 1));
    memcpy(phi_edges, g.ep, sizeof(float) * (g.np + 1));
    ho_geom_free(&g);
    return 0;
}

/* Per-hit admission: slices[n * max_admit] (unused entries = 0xffffffff),
 * count[n].  Returns max_admit. */
int ho_admit_hits(const uint32_t *bins, const float *rng, const float *x, const float *y,
                  const float *z, int64_t n, uint32_t *slices, uint32_t *count)
{
    ho_geom g;
    if (ho_geom_init(&g, bins, rng))
        return -1;
    uint32_t ma = ho_max_admit(&g);
    for (int64_t h = 0; h < n; ++h) {
        uint32_t *o = slices + h * ma;
        for (uint32_t k = 0; k < ma; ++k)
            o[k] = 0xffffffffu;
        count[h] = ho_admit(&g, x[h], y[h], z[h], o);
    }
    ho_geom_free(&g);
    return (int)ma;
}

/* Step 1 (Sec. 2): M[slice][iA][iB] += 1 for every admitted (hit, slice, A
 * bin) whose B falls inside [b_min, b_max).  M must hold
 * n_theta*n_phi*n_a*n_b counters; it is NOT cleared here (accumulates).
 * Returns the number of votes cast. */
int64_t ho_fill(const uint32_t *bins, const float *rng, const float *x, const float *y,
                const float *z, int64_t n, uint32_t *M)
{
    ho_geom g;
    if (ho_geom_init(&g, bins, rng))
        return -1;
    uint32_t *adm = (uint32_t *)malloc(sizeof(uint32_t) * ho_max_admit(&g));
    float nbf = (float)g.nb;
    int64_t votes = 0;
    for (int64_t h = 0; h < n; ++h) {
        float xh = x[h], yh = y[h];
        uint32_t na = ho_admit(&g, xh, yh, z[h], adm);
        if (!na)
            continue;
        float r2 = xh * xh + yh * yh;       /* x^2 + y^2 */
        float d = 2.0f * yh;                 /* 2y */
        for (uint32_t k = 0; k < na; ++k) {
            uint64_t base = (uint64_t)adm[k] * g.na * g.nb;
            for (uint32_t i = 0; i < g.na; ++i) {
                float A = g.a_min + ((float)i + 0.5f) * g.da;   /* A bin centre */
                float twoA = 2.0f * A;
                float num = r2 - twoA * xh;                      /* x^2+y^2-2Ax */
                float B = num / d;                               /* circle centre B */
                float t = (B - g.b_min) / g.db;
                if (t >= 0.0f && t < nbf) {
                    uint32_t j = (uint32_t)t;                    /* floor, t >= 0 */
                    M[base + (uint64_t)i * g.nb + j] += 1u;
                    ++votes;
                }
            }
        }
    }
    free(adm);
    ho_geom_free(&g);
    return votes;
}

/* Step 1 restricted to the slices sel[0..n_sel): Msel[k] is the n_a x n_b
 * matrix of slice sel[k] (accumulated into, not cleared); Msel == NULL only
 * counts.  The loops are those of ho_fill; votes for other slices are not
 * cast.  Returns the number of votes cast into the selected slices. */
int64_t ho_fill_slices(const uint32_t *bins, const float *rng, const float *x, const float *y,
                       const float *z, int64_t n, const uint32_t *sel, int64_t n_sel, uint32_t *Msel)
{
    ho_geom g;
    if (ho_geom_init(&g, bins, rng))
        return -1;
    uint32_t *adm = (uint32_t *)malloc(sizeof(uint32_t) * ho_max_admit(&g));
    float nbf = (float)g.nb;
    int64_t votes = 0;
    for (int64_t h = 0; h < n; ++h) {
        float xh = x[h], yh = y[h];
        uint32_t na = ho_admit(&g, xh, yh, z[h], adm);
        for (uint32_t k = 0; k < na; ++k) {
            int64_t which = -1;
            for (int64_t q = 0; q < n_sel; ++q)
                if (sel[q] == adm[k]) { which = q; break; }
            if (which < 0)
                continue;
            float r2 = xh * xh + yh * yh;
            float d = 2.0f * yh;
            for (uint32_t i = 0; i < g.na; ++i) {
                float A = g.a_min + ((float)i + 0.5f) * g.da;
                float twoA = 2.0f * A;
                float num = r2 - twoA * xh;
                float B = num / d;
                float t = (B - g.b_min) / g.db;
                if (t >= 0.0f && t < nbf) {
                    if (Msel)
                        Msel[(uint64_t)which * g.na * g.nb + (uint64_t)i * g.nb + (uint32_t)t] += 1u;
                    ++votes;
                }
            }
        }
    }
    free(adm);
    ho_geom_free(&g);
    return votes;
}

/* Step 2 (Sec. 2, Sec. 3): threshold + local maxima with the tie rule R7.
 * Writes up to cap peaks in ascending linear index:
 *   ids[5*k .. 5*k+4] = {itheta, iphi, ia, ib, votes}
 *   cen[2*k .. 2*k+1] = {A centre, B centre}
 * Returns the total number of peaks (may exceed cap). */
int64_t ho_find_maxima(const uint32_t *bins, const float *rng, const uint32_t *M,
                       uint32_t threshold, uint32_t *ids, float *cen, int64_t cap)
{
    ho_geom g;
    if (ho_geom_init(&g, bins, rng))
        return -1;
    int64_t found = 0;
    uint64_t ns = (uint64_t)g.nt * g.np;
    for (uint64_t s = 0; s < ns; ++s) {
        const uint32_t *S = M + s * g.na * g.nb;
        for (long i = 0; i < (long)g.na; ++i) {
            for (long j = 0; j < (long)g.nb; ++j) {
                uint32_t v = S[(uint64_t)i * g.nb + j];
                if (v < threshold)
                    continue;
                int peak = 1;
                for (long di = -1; di <= 1 && peak; ++di) {
                    for (long dj = -1; dj <= 1; ++dj) {
                        if (!di && !dj)
                            continue;
                        long ii = i + di, jj = j + dj;
                        if (ii < 0 || ii >= (long)g.na || jj < 0 || jj >= (long)g.nb)
                            continue;
                        uint32_t w = S[(uint64_t)ii * g.nb + jj];
                        /* neighbour before c in linear order: strict */
                        int before = (di < 0) || (di == 0 && dj < 0);
                        if (before ? !(v > w) : !(v >= w)) {
                            peak = 0;
                            break;
                        }
                    }
                }
                if (!peak)
                    continue;
                if (found < cap) {
                    uint32_t *o = ids + 5 * found;
                    o[0] = (uint32_t)(s / g.np);
                    o[1] = (uint32_t)(s % g.np);
                    o[2] = (uint32_t)i;
                    o[3] = (uint32_t)j;
                    o[4] = v;
                    cen[2 * found] = g.a_min + ((float)i + 0.5f) * g.da;
                    cen[2 * found + 1] = g.b_min + ((float)j + 0.5f) * g.db;
                }
                ++found;
            }
        }
    }
    ho_geom_free(&g);
    return found;
}

/* The 4-D variant of the maxima rule: a cell c with v >= threshold is a peak
 * iff it beats every one of its up to 80 neighbours in (theta, phi, A, B) --
 * the cells whose four indices each differ from c's by at most one, other
 * than c; indices outside the matrix are absent and phi does not wrap --
 * strictly when the neighbour comes before c in linear order, else with
 * >=.  Output as ho_find_maxima. */
int64_t ho_find_maxima4d(const uint32_t *bins, const float *rng, const uint32_t *M,
                         uint32_t threshold, uint32_t *ids, float *cen, int64_t cap)
{
    ho_geom g;
    if (ho_geom_init(&g, bins, rng))
        return -1;
    int64_t found = 0;
    for (long t = 0; t < (long)g.nt; ++t) {
        for (long f = 0; f < (long)g.np; ++f) {
            for (long i = 0; i < (long)g.na; ++i) {
                for (long j = 0; j < (long)g.nb; ++j) {
                    const uint64_t lin = (((uint64_t)t * g.np + f) * g.na + i) * g.nb + j;
                    uint32_t v = M[lin];
                    if (v < threshold)
                        continue;
                    int peak = 1;
                    for (long dt = -1; dt <= 1 && peak; ++dt)
                        for (long df = -1; df <= 1 && peak; ++df)
                            for (long di = -1; di <= 1 && peak; ++di)
                                for (long dj = -1; dj <= 1 && peak; ++dj) {
                                    if (!dt && !df && !di && !dj)
                                        continue;
                                    long tt = t + dt, ff = f + df, ii = i + di, jj = j + dj;
                                    if (tt < 0 || tt >= (long)g.nt || ff < 0 || ff >= (long)g.np || ii < 0 ||
                                        ii >= (long)g.na || jj < 0 || jj >= (long)g.nb)
                                        continue;
                                    uint32_t w = M[(((uint64_t)tt * g.np + ff) * g.na + ii) * g.nb + jj];
                                    int before = dt < 0 || (dt == 0 && (df < 0 || (df == 0 && (di < 0 ||
                                                                                               (di == 0 && dj < 0)))));
                                    if (before ? !(v > w) : !(v >= w))
                                        peak = 0;
                                }
                    if (!peak)
                        continue;
                    if (found < cap) {
                        uint32_t *o = ids + 5 * found;
                        o[0] = (uint32_t)t;
                        o[1] = (uint32_t)f;
                        o[2] = (uint32_t)i;
                        o[3] = (uint32_t)j;
                        o[4] = v;
                        cen[2 * found] = g.a_min + ((float)i + 0.5f) * g.da;
                        cen[2 * found + 1] = g.b_min + ((float)j + 0.5f) * g.db;
                    }
                    ++found;
                }
            }
        }
    }
    ho_geom_free(&g);
    return found;
}

/* FP64 variant of the B-bin rule for every admitted (hit, slice, A bin):
 * counts the candidates, the votes cast in FP32, the votes cast in FP64, the
 * candidates whose bin (or in/out decision) differs, and the largest bin
 * distance among the differing in-range pairs.  stats[5] is filled in that
 * order.  diff_out (if not NULL, capacity diff_cap) receives
 * {hit, ia, bin32, bin64} for each differing pair (bin -1 = dropped). */
int ho_bins_f32_vs_f64(const uint32_t *bins, const float *rng, const float *x,
                       const float *y, const float *z, int64_t n, int64_t *stats,
                       int64_t *diff_out, int64_t diff_cap)
{
    ho_geom g;
    if (ho_geom_init(&g, bins, rng))
        return -1;
    uint32_t *adm = (uint32_t *)malloc(sizeof(uint32_t) * ho_max_admit(&g));
    double da64 = ((double)rng[5] - (double)rng[4]) / (double)g.na;
    double db64 = ((double)rng[7] - (double)rng[6]) / (double)g.nb;
    float nbf = (float)g.nb;
    int64_t cand = 0, v32 = 0, v64 = 0, ndiff = 0, maxd = 0;
    for (int64_t h = 0; h < n; ++h) {
        uint32_t na = ho_admit(&g, x[h], y[h], z[h], adm);
        if (!na)
            continue;
        float xh = x[h], yh = y[h];
        float r2 = xh * xh + yh * yh;
        float d = 2.0f * yh;
        double X = xh, Y = yh;
        for (uint32_t i = 0; i < g.na; ++i) {
            float A = g.a_min + ((float)i + 0.5f) * g.da;
            float twoA = 2.0f * A;
            float num = r2 - twoA * xh;
            float B = num / d;
            float t = (B - g.b_min) / g.db;
            long b32 = (t >= 0.0f && t < nbf) ? (long)(uint32_t)t : -1;
            double A64 = (double)rng[4] + ((double)i + 0.5) * da64;
            double B64 = (X * X + Y * Y - 2.0 * A64 * X) / (2.0 * Y);
            double t64 = (B64 - (double)rng[6]) / db64;
            long b64 = (t64 >= 0.0 && t64 < (double)g.nb) ? (long)floor(t64) : -1;
            cand += na;
            if (b32 >= 0) v32 += na;
            if (b64 >= 0) v64 += na;
            if (b32 != b64) {
                if (diff_out && ndiff < diff_cap) {
                    int64_t *o = diff_out + 4 * ndiff;
                    o[0] = h; o[1] = i; o[2] = b32; o[3] = b64;
                }
                ndiff += na;
                if (b32 >= 0 && b64 >= 0) {
                    long dd = labs(b32 - b64);
                    if (dd > maxd) maxd = dd;
                }
            }
        }
    }
    stats[0] = cand; stats[1] = v32; stats[2] = v64; stats[3] = ndiff; stats[4] = maxd;
    free(adm);
    ho_geom_free(&g);
    return 0;
}
