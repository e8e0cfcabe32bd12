/*
 * FP64 CPU oracle for the LArTPC signal-simulation hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline / reference arm load this file's library.  The CUDA library
 * never links, includes or calls it, and it includes nothing of the CUDA library: the
 * two implementations share no source.
 *
 * What it computes (arXiv 2304.01841, §2, the three steps of the signal simulation):
 *   1. Rasterization: each drifted ionisation-electron group ("depo") becomes a 2D patch
 *      of charge over time ticks x pitch impact sub-bins, typically O(20x20).
 *   2. Scatter-add: the patches are summed onto the plane's wire x tick grid.
 *   3. Convolution with the detector response (done in oracle/convolve.py).
 * The paper states these steps in words only.  The quantitative readings used here
 * (drift + diffusion, +-n sigma windows, erf-difference bin integrals normalised to the
 * depo charge, a binomial-like normal-approximation fluctuation drawn from a counter-based
 * Philox4x32-10 stream, folding of impact sub-bins onto wires) are stated beside each
 * function; every one of them is also listed among the readings in the design notes.
 *
 * Everything is plain loops in double precision, in the order the steps are defined.
 * Compile with -ffp-contract=off: the window bounds are decided in FP64 and the GPU path
 * evaluates the same expressions with explicitly rounded FP64 operations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* -------------------------------------------------------------------------------------
 * Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and Shaw
 * ("Parallel random numbers: as easy as 1, 2, 3", SC'11), the Random123 family that the
 * paper's CPU build uses for its RNG (§4.1).  One round maps the counter (c0,c1,c2,c3)
 * with key (k0,k1) through two 32x32->64 multiplications:
 *     (hi0,lo0) = M0*c0,  (hi1,lo1) = M1*c2
 *     c' = (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
 * and between rounds the key is bumped by the Weyl constants (W0, W1).  Ten rounds.
 * ------------------------------------------------------------------------------------- */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += OR_PHILOX_W0;
            k1 += OR_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Batch form for tests: n counters (4 words each) under one key. */
void or_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i)
        or_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0)))
        --q;
    return q;
}

/*
 * The normal deviate of one patch bin (fluctuation pool, counter-based, keyed by absolute
 * bin coordinates so that it does not depend on the order of evaluation):
 *   impact bin j (absolute, may be negative) = wire*n_imp + sub, sub in [0, n_imp)
 *   group g = sub / 4, lane = sub % 4, G = ceil(n_imp / 4)
 *   counter = (depo index, (uint32)tick, (uint32)(wire*G + g), plane<<24 | (event_id & 0xFFFFFF))
 *   key     = (seed low word, seed high word)
 * The four 32-bit outputs become uniforms u = (x + 0.5) * 2^-32 in (0,1); lanes 0,1 are
 * the Box-Muller pair of (u0,u1) and lanes 2,3 the pair of (u2,u3):
 *   r = sqrt(-2 ln u_a),  z_a = r cos(2 pi u_b),  z_b = r sin(2 pi u_b).
 */
double or_bin_normal(uint64_t seed, uint32_t depo_index, int64_t tick, int64_t impact, int32_t n_imp,
                     int32_t plane, uint64_t event_id)
{
    const int64_t G = (n_imp + 3) / 4;
    int64_t wire = floor_div(impact, n_imp);
    int64_t sub = impact - wire * n_imp;
    int64_t g = sub / 4, lane = sub % 4;
    uint32_t ctr[4], key[2], x[4];
    ctr[0] = depo_index;
    ctr[1] = (uint32_t)(int32_t)tick;
    ctr[2] = (uint32_t)(int32_t)(wire * G + g);
    ctr[3] = ((uint32_t)plane << 24) | (uint32_t)(event_id & 0xFFFFFFu);
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, x);
    const double two32 = 4294967296.0;
    int a = (lane < 2) ? 0 : 2;
    double ua = ((double)x[a] + 0.5) / two32;
    double ub = ((double)x[a + 1] + 0.5) / two32;
    double r = sqrt(-2.0 * log(ua));
    const double two_pi = 6.283185307179586476925286766559;
    return (lane % 2 == 0) ? r * cos(two_pi * ub) : r * sin(two_pi * ub);
}

/* -------------------------------------------------------------------------------------
 * Step 1a: drift and diffusion of one depo (standard LArTPC drift-diffusion; the paper's
 * "individual ionization electron groups", §2, binned after drifting to the wires).
 *   t_d   = x / v                      drift time (us)
 *   arrival = t0 + t_d
 *   sigma_L = sqrt(2 D_L t_d),  sigma_T = sqrt(2 D_T t_d)       (mm; D in mm^2/us)
 *   time axis, in tick units:  mu_t = (arrival - t_window0) / tick,
 *                              s_t  = (sigma_L / v) / tick
 *   pitch axis, in impact-bin units (bin width pitch / n_imp):
 *                              p    = z cos(angle) + y sin(angle)
 *                              mu_p = (p - origin) / (pitch / n_imp),  s_p = sigma_T / (pitch / n_imp)
 * Window (reading of "patches span +-n sigma"): the bins overlapping [mu - n s, mu + n s],
 * lo = floor(mu - n s), hi = floor(mu + n s), counted before any clipping to the grid.
 * A width below 1e-6 bin is a point charge: the single bin floor(mu) (an edge belongs to
 * the bin above it).
 * A depo is invalid (skipped, counted) if a coordinate or charge is not finite, x < 0,
 * q < 0, its window exceeds max_nt ticks or max_np impact bins, or the window starts more
 * than 2^30 bins from the origin.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    double mu_t, s_t, mu_p, s_p;
    int64_t lo_t, n_t, lo_p, n_p;
} or_window;

static void axis_window(double mu, double s, double nsigma, int64_t *lo, int64_t *n)
{
    if (s < 1e-6) {
        *lo = (int64_t)floor(mu);
        *n = 1;
        return;
    }
    double a = mu - nsigma * s;
    double b = mu + nsigma * s;
    int64_t l = (int64_t)floor(a), h = (int64_t)floor(b);
    *lo = l;
    *n = h - l + 1;
}

static int depo_window(float t0f, float xf, float yf, float zf, float qf,
                       const double *plane, const double *diff, int64_t max_nt, int64_t max_np,
                       or_window *w)
{
    /* plane = {pitch_mm, origin_mm, angle_rad, tick_us, t_window0_us, n_imp}
       diff  = {DL_cm2_s, DT_cm2_s, v_mm_us, nsigma} */
    double t0 = t0f, x = xf, y = yf, z = zf, q = qf;
    if (!isfinite(t0) || !isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(q))
        return -1;
    if (x < 0.0 || q < 0.0)
        return -1;
    const double pitch = plane[0], origin = plane[1], angle = plane[2];
    const double tick = plane[3], tw0 = plane[4], n_imp = plane[5];
    const double DL = diff[0] * 1.0e-4;     /* cm^2/s -> mm^2/us */
    const double DT = diff[1] * 1.0e-4;
    const double v = diff[2], nsigma = diff[3];

    double t_d = x / v;
    double arrival = t0 + t_d;
    double sigL = sqrt(2.0 * DL * t_d);
    double sigT = sqrt(2.0 * DT * t_d);
    w->mu_t = (arrival - tw0) / tick;
    w->s_t = (sigL / v) / tick;
    double p = z * cos(angle) + y * sin(angle);
    double dp = pitch / n_imp;
    w->mu_p = (p - origin) / dp;
    w->s_p = sigT / dp;
    const double big = 1099511627776.0;   /* 2^40 bins: keeps floor() within int64 */
    if (!(fabs(w->mu_t) < big && fabs(w->mu_p) < big && w->s_t < big && w->s_p < big))
        return -1;
    axis_window(w->mu_t, w->s_t, nsigma, &w->lo_t, &w->n_t);
    axis_window(w->mu_p, w->s_p, nsigma, &w->lo_p, &w->n_p);
    if (w->n_t > max_nt || w->n_p > max_np)
        return -1;
    /* windows more than 2^30 bins from the origin are outside any representable grid */
    const int64_t lim = (int64_t)1 << 30;
    if (w->lo_t < -lim || w->lo_t > lim || w->lo_p < -lim || w->lo_p > lim)
        return -1;
    return 0;
}

/*
 * Step 1b: 1D bin weights (reading of the paper's rasterization into patches, §2):
 * the Gaussian's integral over each window bin, w[i] = (erf(e_{i+1}) - erf(e_i)) / 2 with
 * e = (edge - mu) / (sqrt(2) s), then normalised so the window's weights sum to 1
 * (the patch then carries exactly the depo charge).  Point charge: w = {1}.
 */
static void axis_weights(double mu, double s, int64_t lo, int64_t n, double *w)
{
    if (s < 1e-6) {
        w[0] = 1.0;
        return;
    }
    const double inv = 1.0 / (sqrt(2.0) * s);
    double sum = 0.0;
    double prev = erf(((double)lo - mu) * inv);
    for (int64_t i = 0; i < n; ++i) {
        double e = erf(((double)(lo + i + 1) - mu) * inv);
        w[i] = 0.5 * (e - prev);
        prev = e;
        sum += w[i];
    }
    for (int64_t i = 0; i < n; ++i)
        w[i] /= sum;
}

/* Exposed for tests: the weights of one axis window. */
void or_axis_weights(double mu, double s, double nsigma, int64_t *lo, int64_t *n, double *w, int64_t cap)
{
    axis_window(mu, s, nsigma, lo, n);
    if (*n <= cap)
        axis_weights(mu, s, *lo, *n, w);
}

/*
 * Window pass.  desc[i] = {offset, lo_t, lo_p, n_t, n_p}; offsets are the exclusive prefix
 * sum of n_t*n_p (the paper's patch-offset scan, §4.3).  An invalid depo gets n_t = n_p = 0.
 * mu/s (may be NULL) receive {mu_t, s_t, mu_p, s_p} per depo.  Returns the number of
 * invalid depos; *total_bins receives the patch-buffer size.
 */
int64_t or_windows(int64_t n, const float *t0, const float *x, const float *y, const float *z,
                   const float *q, const double *plane, const double *diff, int64_t max_nt,
                   int64_t max_np, int64_t *desc, double *mus, int64_t *total_bins)
{
    int64_t bad = 0, off = 0;
    for (int64_t i = 0; i < n; ++i) {
        or_window w;
        int64_t *d = desc + 5 * i;
        if (depo_window(t0[i], x[i], y[i], z[i], q[i], plane, diff, max_nt, max_np, &w) != 0) {
            ++bad;
            d[0] = off; d[1] = 0; d[2] = 0; d[3] = 0; d[4] = 0;
            if (mus) { mus[4*i] = mus[4*i+1] = mus[4*i+2] = mus[4*i+3] = 0.0; }
            continue;
        }
        d[0] = off; d[1] = w.lo_t; d[2] = w.lo_p; d[3] = w.n_t; d[4] = w.n_p;
        if (mus) { mus[4*i] = w.mu_t; mus[4*i+1] = w.s_t; mus[4*i+2] = w.mu_p; mus[4*i+3] = w.s_p; }
        off += w.n_t * w.n_p;
    }
    *total_bins = off;
    return bad;
}

/*
 * Rasterization pass (steps 1b + fluctuation), given the windows from or_windows.
 * Patch of depo i, row-major [tick][impact] at patches[desc.offset]:
 *   P[a][b] = q * w_t[a] * w_p[b].
 * With fluctuation (reading of the "binomial-like" charge fluctuation): each bin is the
 * normal approximation to Binomial(n = q, p = w), w = w_t[a] w_p[b],
 *   P'[a][b] = max(0, q w + sqrt(q w (1 - w)) z),  z = or_bin_normal(...)
 * and the patch is rescaled so that it again sums to q (if the fluctuated sum is zero the
 * unfluctuated patch is kept).  The depo index in the counter is the depo's position in
 * the event's arrays.
 */
/* Depo i's patch (the body of or_rasterize's loop); 0, or < 0 on an error. */
static int rasterize_one(int64_t i, const float *t0, const float *x, const float *y, const float *z,
                         const float *q, const double *plane, const double *diff, const int64_t *desc,
                         int32_t fluctuate, uint64_t seed, int32_t plane_index, uint64_t event_id,
                         double *patches)
{
    const int32_t n_imp = (int32_t)plane[5];
    const int64_t *d = desc + 5 * i;
    const int64_t off = d[0], lo_t = d[1], lo_p = d[2], n_t = d[3], n_p = d[4];
    if (n_t == 0 || n_p == 0)
        return 0;
    or_window w;
    if (depo_window(t0[i], x[i], y[i], z[i], q[i], plane, diff, 1 << 30, 1 << 30, &w) != 0)
        return -1;
    double *wt = (double *)malloc(sizeof(double) * (size_t)n_t);
    double *wp = (double *)malloc(sizeof(double) * (size_t)n_p);
    if (!wt || !wp) { free(wt); free(wp); return -2; }
    axis_weights(w.mu_t, w.s_t, lo_t, n_t, wt);
    axis_weights(w.mu_p, w.s_p, lo_p, n_p, wp);
    const double Q = (double)q[i];
    double *P = patches + off;
    for (int64_t a = 0; a < n_t; ++a)
        for (int64_t b = 0; b < n_p; ++b)
            P[a * n_p + b] = Q * wt[a] * wp[b];
    if (fluctuate) {
        double *F = (double *)malloc(sizeof(double) * (size_t)(n_t * n_p));
        if (!F) { free(wt); free(wp); return -2; }
        double sum = 0.0;
        for (int64_t a = 0; a < n_t; ++a) {
            for (int64_t b = 0; b < n_p; ++b) {
                double wb = wt[a] * wp[b];
                double mean = Q * wb;
                double sd = sqrt(Q * wb * (1.0 - wb));
                double zz = or_bin_normal(seed, (uint32_t)i, lo_t + a, lo_p + b, n_imp,
                                          plane_index, event_id);
                double v = mean + sd * zz;
                F[a * n_p + b] = v > 0.0 ? v : 0.0;
                sum += F[a * n_p + b];
            }
        }
        if (sum > 0.0) {
            for (int64_t k = 0; k < n_t * n_p; ++k)
                P[k] = F[k] * (Q / sum);
        }
        free(F);
    }
    free(wt);
    free(wp);
    return 0;
}

int or_rasterize(int64_t n, const float *t0, const float *x, const float *y, const float *z,
                 const float *q, const double *plane, const double *diff, const int64_t *desc,
                 int32_t fluctuate, uint64_t seed, int32_t plane_index, uint64_t event_id,
                 double *patches)
{
    for (int64_t i = 0; i < n; ++i) {
        const int rc = rasterize_one(i, t0, x, y, z, q, plane, diff, desc, fluctuate, seed, plane_index, event_id,
                                     patches);
        if (rc != 0)
            return rc;
    }
    return 0;
}

/*
 * Scatter-add (§2 step 2): every patch bin whose tick lies in [0, n_ticks) and whose
 * impact bin folds (j // n_imp) onto a wire in [0, n_wires) is added to grid[wire][tick]
 * (row-major, ticks fastest).  Bins outside the grid are dropped.
 */
void or_scatter(int64_t n, const int64_t *desc, const double *patches, int32_t n_imp,
                int64_t n_wires, int64_t n_ticks, double *grid)
{
    for (int64_t i = 0; i < n; ++i) {
        const int64_t *d = desc + 5 * i;
        const int64_t off = d[0], lo_t = d[1], lo_p = d[2], n_t = d[3], n_p = d[4];
        for (int64_t a = 0; a < n_t; ++a) {
            int64_t tick = lo_t + a;
            if (tick < 0 || tick >= n_ticks)
                continue;
            for (int64_t b = 0; b < n_p; ++b) {
                int64_t wire = floor_div(lo_p + b, n_imp);
                if (wire < 0 || wire >= n_wires)
                    continue;
                grid[wire * n_ticks + tick] += patches[off + a * n_p + b];
            }
        }
    }
}

/* -------------------------------------------------------------------------------------
 * All-core variants, for timing the oracle on every host core (built with OpenMP when the
 * compiler has it; otherwise they run on one thread).  They compute exactly what the serial
 * functions above compute:
 *   or_rasterize_omp: depos spread over the threads (each patch is written by one thread,
 *     at its own offset), so the patches are bit-identical to or_rasterize's;
 *   or_scatter_omp: each thread owns a band of wires and adds, in depo order, the bins of
 *     every patch that fold onto its band, so every bin's sum is taken in the serial order
 *     and the grid is bit-identical to or_scatter's (no per-thread grid copies, no reduction).
 * n_threads <= 0: the OpenMP default.  or_omp_threads reports the threads they will use.
 * ------------------------------------------------------------------------------------- */
#ifdef _OPENMP
#include <omp.h>
#endif

int32_t or_omp_threads(int32_t n_threads)
{
#ifdef _OPENMP
    return n_threads > 0 ? n_threads : (int32_t)omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

int or_rasterize_omp(int64_t n, const float *t0, const float *x, const float *y, const float *z,
                     const float *q, const double *plane, const double *diff, const int64_t *desc,
                     int32_t fluctuate, uint64_t seed, int32_t plane_index, uint64_t event_id,
                     double *patches, int32_t n_threads)
{
    int err = 0;
    const int nt = or_omp_threads(n_threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt) reduction(min : err)
    for (int64_t i = 0; i < n; ++i) {
        const int rc = rasterize_one(i, t0, x, y, z, q, plane, diff, desc, fluctuate, seed, plane_index, event_id,
                                     patches);
        if (rc < err)
            err = rc;
    }
    return err;
}

void or_scatter_omp(int64_t n, const int64_t *desc, const double *patches, int32_t n_imp,
                    int64_t n_wires, int64_t n_ticks, double *grid, int32_t n_threads)
{
    const int nt = or_omp_threads(n_threads);
    (void)nt;
#pragma omp parallel num_threads(nt)
    {
        int T = 1, me = 0;
#ifdef _OPENMP
        T = omp_get_num_threads();
        me = omp_get_thread_num();
#endif
        const int64_t w_lo = n_wires * me / T, w_hi = n_wires * (me + 1) / T;   /* this thread's band */
        for (int64_t i = 0; i < n; ++i) {
            const int64_t *d = desc + 5 * i;
            const int64_t off = d[0], lo_t = d[1], lo_p = d[2], n_t = d[3], n_p = d[4];
            if (n_t == 0 || n_p == 0)
                continue;
            if (floor_div(lo_p + n_p - 1, n_imp) < w_lo || floor_div(lo_p, n_imp) >= w_hi)
                continue;                                  /* no bin of this patch in the band */
            for (int64_t a = 0; a < n_t; ++a) {
                int64_t tick = lo_t + a;
                if (tick < 0 || tick >= n_ticks)
                    continue;
                for (int64_t b = 0; b < n_p; ++b) {
                    int64_t wire = floor_div(lo_p + b, n_imp);
                    if (wire < w_lo || wire >= w_hi)
                        continue;
                    grid[wire * n_ticks + tick] += patches[off + a * n_p + b];
                }
            }
        }
    }
}

/*
 * Direct linear convolution (§2 step 3, written out): with the response centred in wire
 * (row kc = n_wr/2 is the wire the charge sits on) and causal in time,
 *   out[w][t] = sum_{r=0}^{n_wr-1} sum_{tau=0}^{n_tr-1} grid[w - (r - kc)][t - tau] * resp[r][tau]
 * with the grid zero outside [0,n_wires) x [0,n_ticks); the output covers the grid.
 * Literal quadruple loop: only for small grids.
 */
void or_convolve_direct(const double *grid, int64_t n_wires, int64_t n_ticks, const double *resp,
                        int64_t n_wr, int64_t n_tr, double *out)
{
    const int64_t kc = n_wr / 2;
    for (int64_t w = 0; w < n_wires; ++w) {
        for (int64_t t = 0; t < n_ticks; ++t) {
            double acc = 0.0;
            for (int64_t r = 0; r < n_wr; ++r) {
                int64_t ws = w - (r - kc);
                if (ws < 0 || ws >= n_wires)
                    continue;
                for (int64_t tau = 0; tau < n_tr; ++tau) {
                    int64_t ts = t - tau;
                    if (ts < 0 || ts >= n_ticks)
                        continue;
                    acc += grid[ws * n_ticks + ts] * resp[r * n_tr + tau];
                }
            }
            out[w * n_ticks + t] = acc;
        }
    }
}
