/*
 * FP64 oracle of the Monte Carlo line-transfer pass (plain C).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this library. The product path never does.
 * It shares no code with the CUDA path: its own Philox generator, its own
 * cell walk, scattering and tallies, fed with tables built by
 * oracle/tables.py from the paper's definitions.
 *
 * One packet at a time, one event at a time, in the order the method takes
 * its steps:
 *   emission (Sec. 2.1: isotropic, line centre or thermal profile; Sec. 3),
 *   free path tau = -ln(xi),
 *   cell walk with alpha = alpha0 H(a, x_com) in the comoving frame
 *     (Sec. 2.1, Eq. xdef, Sec. 2.2.1 bulk-velocity projection),
 *   scattering (Sec. 2.1.2, Eq. riia-scatter) with u_par from the velocity
 *     sampler (Sec. 2.1.1), isotropic re-emission, destruction with
 *     probability epsilon (Eq. eps),
 *   per-segment tallies: excitation (Sec. 2.1.3 pumping rate), comoving
 *     channel path length (mean intensity), camera-directed scattering
 *     emissivity (Eq. scat-line with Eq. riia-table / riia-inf),
 *   continuum (dust) absorption: the packet weight decays as exp(-dtau_e)
 *     along each segment and the segment's tallies take the mean weight
 *     (1 - exp(-dtau_e))/dtau_e (Eq. scat-line); the absorbed weight is
 *     tallied per cell and a packet below the weight cut ends as absorbed,
 *   escape into the lab-frame spectrum (Sec. 2.3.2) with the packet weight.
 *
 * Precision model: the per-cell fields and the tables arrive already
 * rounded to float32 (the method stores them in single precision, Sec. 2.3);
 * every operation here is FP64.
 *
 * Random numbers: Philox4x32-10 (Salmon et al. 2011) with counter
 * (packet_lo, packet_hi, event, block) and key (seed_lo, seed_hi). A 32-bit
 * output r maps to the uniform ((r >> 9) + 1/2) 2^-23, which lies in
 * [2^-24, 1 - 2^-24] and is exact in both FP32 and FP64. Slot map:
 *   emission (event 0): block 0 = {mu, phi, tau, freq1}
 *                       block 1 = {freq2, pos_a, pos_b, pos_c}
 *                       block 2 = {cell_hi, cell_lo, -, -} (volume source)
 *   scattering (event e >= 1): block 0 = {u_par, bm_radius, bm_angle, tau}
 *                              block 1 = {mu, phi, eps_test, -}
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

enum { ORC_SRC_POINT = 0, ORC_SRC_PLANE = 1, ORC_SRC_BEAM = 2, ORC_SRC_VOLUME = 3 };
enum { ORC_PROFILE_LINE_CENTRE = 0, ORC_PROFILE_GAUSSIAN = 1 };
enum { ORC_T_SCATMAP = 1, ORC_T_EXC = 2, ORC_T_J = 4, ORC_T_EMISS = 8 };
enum { ORC_ESCAPED = 1, ORC_DESTROYED = 2, ORC_STUCK = 3, ORC_ABSORBED = 4 };

/* table geometry (fixed by the readings in oracle/tables.py) */
#define V_N 5000
#define V_LMIN (-4.0)
#define V_LMAX 3.0
#define US_NX 40
#define US_NU 251
#define US_UMIN (-6.0)
#define US_DU 0.048
#define R_ND 201
#define R_NX 200
#define R_NG 40
#define R_DMAX 10.0
#define R_DSTEP 0.1
#define R_XMAX 120.0
#define R_SMIN 0.1

typedef struct {
    int nx, ny, nz;
    int periodic[3];
    const double* tau0;      /* [ncell] line-centre optical depth per cell width */
    const double* vel;       /* [ncell][3] bulk velocity in units of b, or NULL */
    const double* eps;       /* [ncell] destruction probability, or NULL */
    double a;
    const double* voigt_lnH; /* [5000] */
    double voigt_H0;
    const double* us_x;      /* [40] */
    const double* us_lncdf;  /* [40][251] */
    const double* rtab;      /* [40][200][201], needed for the emissivity tally */
    int src_kind;
    double src_pos[3];
    int src_axis;
    double src_plane;
    int band_axis;
    double band_lo, band_hi;
    int src_profile;
    const double* src_cdf;   /* [ncell] inclusive cumulative emission weights, last = 1 */
    double spec_lo, spec_hi;
    int spec_n;
    int n_ch;
    double ch_x0, ch_dx;     /* channel k spans velocities [v_min + k dv, v_min + (k+1) dv),
                                velocity v <-> x = -v / b; x0 = v_min / b, dx = dv / b */
    int n_cam;
    const double* cam_dir;   /* [n_cam][3] unit propagation directions toward cameras */
    unsigned tally_flags;
    uint64_t max_iters;      /* per-packet cap on walk iterations */
    int ph_mode;             /* 2: the 1-D slice; 1: the 2-D table; 3: core-wing blend */
    const double* voigt2d;   /* [64][512] ln H for ph_mode 1 */
    double u0;               /* core-wing crossing point for ph_mode 3 */
    const double* tau_abs;   /* [ncell] continuum absorption optical depth per cell width, or NULL */
    double wcut;             /* a packet whose weight falls below this is absorbed */
} orc_problem;

typedef struct {
    double x;                /* lab-frame x at termination */
    uint32_t nscat;
    uint32_t ncross;
    uint32_t status;
    uint32_t cell0;          /* flat index of the emission cell */
} orc_record;

typedef struct {
    double* spec_w;          /* [spec_n + 2]: underflow, bins, overflow */
    uint64_t* spec_c;        /* [spec_n + 2] */
    uint64_t* scat;          /* [ncell] */
    double* exc;             /* [ncell]     sum of w ds H(a, x_com) */
    double* J;               /* [ncell][n_ch] sum of w ds in the comoving channel of x_com */
    double* emiss;           /* [n_cam][ncell][n_ch] */
    double* absw;            /* [ncell] packet weight absorbed by the continuum */
    uint64_t stats[8];       /* emitted, escaped, destroyed, stuck, scatterings, crossings,
                                absorbed (weight below wcut) */
    orc_record* rec;         /* [n] or NULL */
} orc_tallies;

/* ------------------------------------------------------------ Philox4x32-10 */

static void philox4x32_10(const uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static double u01(uint32_t r) { return (double)(r >> 9) * (1.0 / 8388608.0) + (1.0 / 16777216.0); }

typedef struct { uint32_t k0, k1, p0, p1; } rng_ctx;

static void draw(const rng_ctx* g, uint32_t event, uint32_t block, double u[4], uint32_t raw[4])
{
    uint32_t c[4] = { g->p0, g->p1, event, block };
    uint32_t o[4];
    philox4x32_10(c, g->k0, g->k1, o);
    for (int i = 0; i < 4; ++i) {
        if (u) u[i] = u01(o[i]);
        if (raw) raw[i] = o[i];
    }
}

/* exported for the tests: raw Philox words */
void orc_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, int n)
{
    for (int i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, k0, k1, out + 4 * i);
}

/* ------------------------------------------------------------ profile, sampler, kernel */

/* ph_mode 1 (Sec. 2.3.1): bilinear lookup of ln H in (log10 a, log10|x|)
 * on the two-dimensional table; a nodes uniform in log10 a over [-6, 0]
 * (64), x nodes uniform in log10|x| over [-4, 3] (512). */
#define V2_NA 64
#define V2_NX 512
#define V2_LA_MIN (-6.0)
#define V2_LA_MAX 0.0

static double voigt2d_lookup(const orc_problem* P, double ax)
{
    if (ax > 1e3) return P->a / (sqrt(ORC_PI) * ax * ax) * (1.0 + 1.5 / (ax * ax));
    double s = (log10(P->a) - V2_LA_MIN) * ((V2_NA - 1) / (V2_LA_MAX - V2_LA_MIN));
    int j = (int)floor(s);
    if (j < 0) j = 0;
    if (j > V2_NA - 2) j = V2_NA - 2;
    double w = s - j;
    double t = (log10(ax < 1e-4 ? 1e-4 : ax) - V_LMIN) * ((V2_NX - 1) / (V_LMAX - V_LMIN));
    if (t < 0.0) t = 0.0;
    int i = (int)floor(t);
    if (i > V2_NX - 2) i = V2_NX - 2;
    double f = t - i;
    const double* r0 = P->voigt2d + (size_t)j * V2_NX;
    const double* r1 = r0 + V2_NX;
    double l0 = (1.0 - f) * r0[i] + f * r0[i + 1];
    double l1 = (1.0 - f) * r1[i] + f * r1[i + 1];
    return exp((1.0 - w) * l0 + w * l1);
}

/* ph_mode 3 (Sec. 2.3.1): (1 - w) exp(-x^2) + w a / (sqrt(pi) (x^2 + a^2))
 * with w = [1 + tanh(2|x| - 2 u0)] / 2 = 1 / (1 + exp(4 (u0 - |x|))). */
static double blend_lookup(const orc_problem* P, double ax)
{
    double w = 1.0 / (1.0 + exp(4.0 * (P->u0 - ax)));
    double core = exp(-ax * ax);
    double wing = P->a / (sqrt(ORC_PI) * (ax * ax + P->a * P->a));
    return (1.0 - w) * core + w * wing;
}

static double voigt_lookup(const orc_problem* P, double x)
{
    double ax = fabs(x);
    if (P->ph_mode == 1) return voigt2d_lookup(P, ax);
    if (P->ph_mode == 3) return blend_lookup(P, ax);
    if (ax < 1e-4) return P->voigt_H0;
    if (ax > 1e3) return P->a / (sqrt(ORC_PI) * ax * ax) * (1.0 + 1.5 / (ax * ax));
    double t = (log10(ax) - V_LMIN) * ((V_N - 1) / (V_LMAX - V_LMIN));
    int i = (int)floor(t);
    if (i < 0) i = 0;
    if (i > V_N - 2) i = V_N - 2;
    double f = t - i;
    return exp((1.0 - f) * P->voigt_lnH[i] + f * P->voigt_lnH[i + 1]);
}

/* largest i in [0, n-2] with v[i] <= t (v ascending), by bisection */
static int bracket(const double* v, int n, double t)
{
    int lo = 0, hi = n - 1;          /* invariant: answer in [lo, hi-1] when v[lo] <= t */
    if (t < v[0]) return 0;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (v[mid] <= t) lo = mid; else hi = mid;
    }
    return lo > n - 2 ? n - 2 : lo;
}

static double us_invert_row(const orc_problem* P, int row, double L)
{
    const double* c = P->us_lncdf + (size_t)row * US_NU;
    int j = bracket(c, US_NU, L);
    return US_UMIN + US_DU * j + US_DU * (L - c[j]) / (c[j + 1] - c[j]);
}

static double us_sample(const orc_problem* P, double x, double xi)
{
    double ax = fabs(x);
    int i = bracket(P->us_x, US_NX, ax);
    double t = (ax - P->us_x[i]) / (P->us_x[i + 1] - P->us_x[i]);
    double L = log(xi);
    double u = (1.0 - t) * us_invert_row(P, i, L) + t * us_invert_row(P, i + 1, L);
    return x < 0.0 ? -u : u;
}

static double r_kernel(const orc_problem* P, double D, double x, double g)
{
    if (x < 0.0) { D = -D; x = -x; }
    if (fabs(D) > R_DMAX) return 0.0;
    if (x >= R_XMAX) {
        double v = 1.0 - g;
        if (v < R_SMIN * R_SMIN) v = R_SMIN * R_SMIN;
        return exp(-D * D / (2.0 * v)) / sqrt(2.0 * ORC_PI * v);
    }
    double fd = (D + R_DMAX) / R_DSTEP;
    double fx = x * (R_NX - 1) / R_XMAX;
    double fg = (g + 1.0) * (R_NG - 1) / 2.0;
    int i = (int)floor(fd), j = (int)floor(fx), k = (int)floor(fg);
    i = i < 0 ? 0 : (i > R_ND - 2 ? R_ND - 2 : i);
    j = j < 0 ? 0 : (j > R_NX - 2 ? R_NX - 2 : j);
    k = k < 0 ? 0 : (k > R_NG - 2 ? R_NG - 2 : k);
    double wd = fd - i, wx = fx - j, wg = fg - k;
    double acc = 0.0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj) {
            const double* row = P->rtab + ((size_t)(k + dk) * R_NX + (j + dj)) * R_ND;
            double c = (dk ? wg : 1.0 - wg) * (dj ? wx : 1.0 - wx);
            acc += c * ((1.0 - wd) * row[i] + wd * row[i + 1]);
        }
    return acc;
}

/* ------------------------------------------------------------ geometry */

static void iso_dir(double mu_u, double phi_u, double n[3])
{
    double mu = 2.0 * mu_u - 1.0;
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double ph = 2.0 * ORC_PI * phi_u;
    n[0] = st * cos(ph);
    n[1] = st * sin(ph);
    n[2] = mu;
}

static double vdot(const orc_problem* P, size_t c, const double n[3])
{
    if (!P->vel) return 0.0;
    const double* v = P->vel + 3 * c;
    return n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
}

typedef struct {
    int ci[3];          /* cell index */
    double p[3];        /* position inside the cell, in [0, 1] */
    double n[3];        /* direction */
    double x;           /* lab-frame frequency in Doppler units */
    double tau;         /* remaining optical depth to the next scattering */
    double w;           /* weight (photon number per packet, unit here) */
} orc_packet;

/* Place a packet at absolute coordinate X (cell units) along each axis; a
   packet sitting on a cell face belongs to the cell it moves into. */
static int place(const orc_problem* P, orc_packet* k, const double X[3])
{
    const int dims[3] = { P->nx, P->ny, P->nz };
    for (int d = 0; d < 3; ++d) {
        double f = floor(X[d]);
        int c = (int)f;
        double p = X[d] - f;
        if (p == 0.0 && k->n[d] < 0.0) { c -= 1; p = 1.0; }
        if (P->periodic[d]) { c %= dims[d]; if (c < 0) c += dims[d]; }
        if (c < 0 || c >= dims[d]) return 0;
        k->ci[d] = c;
        k->p[d] = p;
    }
    return 1;
}

static size_t cell_of(const orc_problem* P, const int ci[3])
{
    return ((size_t)ci[2] * P->ny + ci[1]) * P->nx + ci[0];
}

/* ------------------------------------------------------------ tallies */

static void add_spectrum(const orc_problem* P, orc_tallies* T, double x, double w)
{
    int b;
    if (x < P->spec_lo) b = 0;
    else if (x >= P->spec_hi) b = P->spec_n + 1;
    else {
        b = 1 + (int)floor((x - P->spec_lo) / (P->spec_hi - P->spec_lo) * P->spec_n);
        if (b > P->spec_n) b = P->spec_n;
    }
    T->spec_w[b] += w;
    T->spec_c[b] += 1;
}

/* Continuum absorption over a segment of optical depth dt (Sec. 2.2.1,
 * Eq. scat-line): the packet weight decays as exp(-dt); the segment's
 * tallies take the weight at its start times (1 - exp(-dt)) / dt, the mean
 * weight along it (evaluated as -expm1(-dt)/dt, and by its series below
 * dt = 1e-4). Returns that factor and the absorbed fraction 1 - exp(-dt). */
static double segment_factor(double dt, double* absorbed)
{
    *absorbed = -expm1(-dt);
    if (dt < 1e-4) return 1.0 - dt * (0.5 - dt * (1.0 / 6.0 - dt / 24.0));
    return *absorbed / dt;
}

static void tally_segment(const orc_problem* P, orc_tallies* T, size_t c, const orc_packet* k,
                          double ds, double xcom, double H, double fseg)
{
    unsigned f = P->tally_flags;
    size_t ncell = (size_t)P->nx * P->ny * P->nz;
    const double w = k->w * fseg;
    if (f & ORC_T_EXC) T->exc[c] += w * ds * H;
    if ((f & ORC_T_J) && P->n_ch > 0) {
        /* comoving channel of x_com: velocity v = -x b, k = floor((v - vmin) / dv) */
        double q = (-xcom - P->ch_x0) / P->ch_dx;
        if (q >= 0.0 && q < P->n_ch) T->J[c * P->n_ch + (size_t)floor(q)] += w * ds;
    }
    if ((f & ORC_T_EMISS) && P->n_ch > 0) {
        double base = w * ds * P->tau0[c] * H / (4.0 * ORC_PI);
        for (int m = 0; m < P->n_cam; ++m) {
            const double* nc = P->cam_dir + 3 * m;
            double g = k->n[0] * nc[0] + k->n[1] * nc[1] + k->n[2] * nc[2];
            double vc = vdot(P, c, nc);
            for (int ch = 0; ch < P->n_ch; ++ch) {
                /* gas-frame frequency of channel ch seen along nc: -(v_k + nc.V)/b */
                double xout = -(P->ch_x0 + (ch + 0.5) * P->ch_dx) - vc;
                double D = xout - xcom;
                if (fabs(D) > R_DMAX) continue;
                T->emiss[((size_t)m * ncell + c) * P->n_ch + ch] += base * r_kernel(P, D, xcom, g);
            }
        }
    }
}

/* ------------------------------------------------------------ one packet */

static void emit(const orc_problem* P, const rng_ctx* g, orc_packet* k, int* ok)
{
    double b0[4], b1[4];
    uint32_t r2[4];
    draw(g, 0, 0, b0, NULL);
    draw(g, 0, 1, b1, NULL);
    k->w = 1.0;
    double X[3] = { 0, 0, 0 };
    const double dims[3] = { P->nx, P->ny, P->nz };
    if (P->src_kind == ORC_SRC_BEAM) {
        int ax = P->src_axis;
        k->n[0] = k->n[1] = k->n[2] = 0.0;
        k->n[ax] = 1.0;
        double pos[2] = { b1[1], b1[2] };
        int q = 0;
        for (int d = 0; d < 3; ++d) {
            if (d == ax) { X[d] = 0.0; continue; }
            if (d == P->band_axis) X[d] = P->band_lo + (P->band_hi - P->band_lo) * pos[q];
            else X[d] = dims[d] * pos[q];
            ++q;
        }
    } else {
        iso_dir(b0[0], b0[1], k->n);
        if (P->src_kind == ORC_SRC_POINT) {
            for (int d = 0; d < 3; ++d) X[d] = P->src_pos[d];
        } else if (P->src_kind == ORC_SRC_PLANE) {
            int q = 1;
            for (int d = 0; d < 3; ++d) X[d] = (d == P->src_axis) ? P->src_plane : dims[d] * b1[q++];
        } else {
            draw(g, 0, 2, NULL, r2);
            double uc = (double)(r2[0] >> 8) * (1.0 / 16777216.0)
                      + (double)(r2[1] >> 8) * (1.0 / 281474976710656.0)
                      + (1.0 / 562949953421312.0);
            size_t ncell = (size_t)P->nx * P->ny * P->nz;
            /* first cell whose inclusive cumulative weight exceeds uc */
            size_t lo = 0, hi = ncell - 1;
            while (lo < hi) {
                size_t mid = (lo + hi) / 2;
                if (P->src_cdf[mid] > uc) hi = mid; else lo = mid + 1;
            }
            int cz = (int)(lo / ((size_t)P->nx * P->ny));
            int cy = (int)((lo / P->nx) % P->ny);
            int cx = (int)(lo % P->nx);
            X[0] = cx + b1[1];
            X[1] = cy + b1[2];
            X[2] = cz + b1[3];
        }
    }
    *ok = place(P, k, X);
    double xcom = 0.0;
    if (P->src_profile == ORC_PROFILE_GAUSSIAN)
        xcom = sqrt(-log(b0[3])) * cos(2.0 * ORC_PI * b1[0]);
    size_t c = *ok ? cell_of(P, k->ci) : 0;
    k->x = xcom + (*ok ? vdot(P, c, k->n) : 0.0);
    k->tau = -log(b0[2]);
}

static void run_packet(const orc_problem* P, uint64_t id, uint32_t k0, uint32_t k1,
                       orc_tallies* T, orc_record* rec)
{
    rng_ctx g = { k0, k1, (uint32_t)id, (uint32_t)(id >> 32) };
    orc_packet k;
    int ok;
    emit(P, &g, &k, &ok);
    T->stats[0] += 1;
    uint32_t nscat = 0, ncross = 0, status = ORC_STUCK;
    const int dims[3] = { P->nx, P->ny, P->nz };
    uint32_t cell0 = ok ? (uint32_t)cell_of(P, k.ci) : 0xFFFFFFFFu;
    if (!ok) { status = ORC_ESCAPED; add_spectrum(P, T, k.x, k.w); goto done; }
    for (uint64_t it = 0; it < P->max_iters; ++it) {
        size_t c = cell_of(P, k.ci);
        double xcom = k.x - vdot(P, c, k.n);
        double H = voigt_lookup(P, xcom);
        double alpha = P->tau0[c] * H;              /* per cell width */
        /* distance to the cell boundary, ties to the lowest axis */
        double s_exit = INFINITY;
        int axis = -1;
        for (int d = 0; d < 3; ++d) {
            double t;
            if (k.n[d] > 0.0) t = (1.0 - k.p[d]) / k.n[d];
            else if (k.n[d] < 0.0) t = -k.p[d] / k.n[d];
            else continue;
            if (t < s_exit) { s_exit = t; axis = d; }
        }
        if (k.tau < alpha * s_exit) {
            /* scattering inside this cell */
            double s = k.tau / alpha;
            for (int d = 0; d < 3; ++d) k.p[d] = fmin(1.0, fmax(0.0, k.p[d] + s * k.n[d]));
            double fseg = 1.0, fabs_ = 0.0;
            if (P->tau_abs) fseg = segment_factor(P->tau_abs[c] * s, &fabs_);
            tally_segment(P, T, c, &k, s, xcom, H, fseg);
            if (P->tau_abs) {
                T->absw[c] += k.w * fabs_;
                k.w *= 1.0 - fabs_;
                if (k.w < P->wcut) { status = ORC_ABSORBED; break; }
            }
            ++nscat;
            if (P->tally_flags & ORC_T_SCATMAP) T->scat[c] += 1;
            double u0[4], u1[4];
            draw(&g, nscat, 0, u0, NULL);
            draw(&g, nscat, 1, u1, NULL);
            if (P->eps && u1[2] < P->eps[c]) { status = ORC_DESTROYED; break; }
            double rad = sqrt(-log(u0[1]));
            double z1 = rad * cos(2.0 * ORC_PI * u0[2]);
            double z2 = rad * sin(2.0 * ORC_PI * u0[2]);
            double upar = fabs(xcom) > 300.0 ? z2 : us_sample(P, xcom, u0[0]);
            double no[3];
            iso_dir(u1[0], u1[1], no);
            double gg = k.n[0] * no[0] + k.n[1] * no[1] + k.n[2] * no[2];
            double sg = sqrt(fmax(0.0, 1.0 - gg * gg));
            double xout = xcom + upar * (gg - 1.0) + z1 * sg;
            for (int d = 0; d < 3; ++d) k.n[d] = no[d];
            k.x = xout + vdot(P, c, k.n);
            k.tau = -log(u0[3]);
        } else {
            /* cross the face on `axis` */
            k.tau -= alpha * s_exit;
            for (int d = 0; d < 3; ++d) {
                if (d == axis) continue;
                k.p[d] = fmin(1.0, fmax(0.0, k.p[d] + s_exit * k.n[d]));
            }
            double fseg = 1.0, fabs_ = 0.0;
            if (P->tau_abs) fseg = segment_factor(P->tau_abs[c] * s_exit, &fabs_);
            tally_segment(P, T, c, &k, s_exit, xcom, H, fseg);
            if (P->tau_abs) {
                T->absw[c] += k.w * fabs_;
                k.w *= 1.0 - fabs_;
                if (k.w < P->wcut) { status = ORC_ABSORBED; break; }
            }
            ++ncross;
            int step = k.n[axis] > 0.0 ? 1 : -1;
            int nc = k.ci[axis] + step;
            k.p[axis] = step > 0 ? 0.0 : 1.0;
            if (nc < 0 || nc >= dims[axis]) {
                if (!P->periodic[axis]) { status = ORC_ESCAPED; add_spectrum(P, T, k.x, k.w); break; }
                nc = (nc + dims[axis]) % dims[axis];
            }
            k.ci[axis] = nc;
        }
    }
done:
    if (status == ORC_ESCAPED) T->stats[1] += 1;
    else if (status == ORC_DESTROYED) T->stats[2] += 1;
    else if (status == ORC_ABSORBED) T->stats[6] += 1;
    else T->stats[3] += 1;
    T->stats[4] += nscat;
    T->stats[5] += ncross;
    if (rec) { rec->x = k.x; rec->nscat = nscat; rec->ncross = ncross; rec->status = status; rec->cell0 = cell0; }
}

/* ------------------------------------------------------------ threads */

typedef struct {
    const orc_problem* P;
    uint64_t first, count;
    uint32_t k0, k1;
    orc_tallies T;
    orc_record* rec;
} orc_job;

static void* worker(void* arg)
{
    orc_job* j = (orc_job*)arg;
    for (uint64_t i = 0; i < j->count; ++i)
        run_packet(j->P, j->first + i, j->k0, j->k1, &j->T, j->rec ? j->rec + i : NULL);
    return NULL;
}

static void tallies_alloc(const orc_problem* P, orc_tallies* T)
{
    size_t ncell = (size_t)P->nx * P->ny * P->nz;
    unsigned f = P->tally_flags;
    memset(T, 0, sizeof(*T));
    T->spec_w = calloc((size_t)P->spec_n + 2, sizeof(double));
    T->spec_c = calloc((size_t)P->spec_n + 2, sizeof(uint64_t));
    if (f & ORC_T_SCATMAP) T->scat = calloc(ncell, sizeof(uint64_t));
    if (f & ORC_T_EXC) T->exc = calloc(ncell, sizeof(double));
    if (f & ORC_T_J) T->J = calloc(ncell * (size_t)(P->n_ch > 0 ? P->n_ch : 1), sizeof(double));
    if (f & ORC_T_EMISS)
        T->emiss = calloc((size_t)(P->n_cam > 0 ? P->n_cam : 1) * ncell * (size_t)(P->n_ch > 0 ? P->n_ch : 1),
                          sizeof(double));
    if (P->tau_abs) T->absw = calloc(ncell, sizeof(double));
}

static void tallies_free(orc_tallies* T)
{
    free(T->spec_w); free(T->spec_c); free(T->scat); free(T->exc); free(T->J); free(T->emiss); free(T->absw);
}

/*
 * Run packets [first, first + n) with key = (seed_lo, seed_hi) on nthreads
 * threads (contiguous packet ranges, reduced in thread order) and ADD the
 * results into *out. out->rec, if set, receives one record per packet.
 * Returns 0, or -1 on an allocation failure.
 */
int orc_run(const orc_problem* P, uint64_t first, uint64_t n, uint32_t seed_lo, uint32_t seed_hi,
            int nthreads, orc_tallies* out)
{
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > n && n > 0) nthreads = (int)n;
    orc_job* jobs = calloc((size_t)nthreads, sizeof(orc_job));
    pthread_t* th = calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    uint64_t per = nthreads ? n / (uint64_t)nthreads : 0, rem = nthreads ? n % (uint64_t)nthreads : 0;
    uint64_t at = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t cnt = per + ((uint64_t)t < rem ? 1 : 0);
        jobs[t].P = P;
        jobs[t].first = first + at;
        jobs[t].count = cnt;
        jobs[t].k0 = seed_lo;
        jobs[t].k1 = seed_hi;
        jobs[t].rec = out->rec ? out->rec + at : NULL;
        tallies_alloc(P, &jobs[t].T);
        at += cnt;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, &jobs[t]);
    worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);

    size_t ncell = (size_t)P->nx * P->ny * P->nz;
    unsigned f = P->tally_flags;
    for (int t = 0; t < nthreads; ++t) {
        orc_tallies* T = &jobs[t].T;
        for (int b = 0; b < P->spec_n + 2; ++b) { out->spec_w[b] += T->spec_w[b]; out->spec_c[b] += T->spec_c[b]; }
        if (f & ORC_T_SCATMAP) for (size_t c = 0; c < ncell; ++c) out->scat[c] += T->scat[c];
        if (f & ORC_T_EXC) for (size_t c = 0; c < ncell; ++c) out->exc[c] += T->exc[c];
        if (P->tau_abs && out->absw) for (size_t c = 0; c < ncell; ++c) out->absw[c] += T->absw[c];
        if (f & ORC_T_J) for (size_t c = 0; c < ncell * (size_t)P->n_ch; ++c) out->J[c] += T->J[c];
        if (f & ORC_T_EMISS)
            for (size_t c = 0; c < (size_t)P->n_cam * ncell * (size_t)P->n_ch; ++c) out->emiss[c] += T->emiss[c];
        for (int s = 0; s < 8; ++s) out->stats[s] += T->stats[s];
        tallies_free(T);
    }
    free(jobs);
    free(th);
    return 0;
}

/*
 * Cell walk alone, for the geometry tests: follow a ray from absolute
 * position X (cell units) along unit direction n through an opacity-free
 * grid until it leaves the domain or max_seg segments are written; writes
 * the visited flat cell index and segment length per segment. Returns the
 * number of segments.
 */
int orc_trace(const orc_problem* P, const double* X, const double* n, int max_seg,
              int64_t* cells, double* lens)
{
    orc_packet k;
    memset(&k, 0, sizeof(k));
    for (int d = 0; d < 3; ++d) k.n[d] = n[d];
    if (!place(P, &k, X)) return 0;
    const int dims[3] = { P->nx, P->ny, P->nz };
    int ns = 0;
    while (ns < max_seg) {
        double s_exit = INFINITY;
        int axis = -1;
        for (int d = 0; d < 3; ++d) {
            double t;
            if (k.n[d] > 0.0) t = (1.0 - k.p[d]) / k.n[d];
            else if (k.n[d] < 0.0) t = -k.p[d] / k.n[d];
            else continue;
            if (t < s_exit) { s_exit = t; axis = d; }
        }
        cells[ns] = (int64_t)cell_of(P, k.ci);
        lens[ns] = s_exit;
        ++ns;
        for (int d = 0; d < 3; ++d)
            if (d != axis) k.p[d] = fmin(1.0, fmax(0.0, k.p[d] + s_exit * k.n[d]));
        int step = k.n[axis] > 0.0 ? 1 : -1;
        int nc = k.ci[axis] + step;
        k.p[axis] = step > 0 ? 0.0 : 1.0;
        if (nc < 0 || nc >= dims[axis]) {
            if (!P->periodic[axis]) break;
            nc = (nc + dims[axis]) % dims[axis];
        }
        k.ci[axis] = nc;
    }
    return ns;
}

/* exported for the tests: sampler and kernel lookups as the walk uses them */
double orc_us_sample(const orc_problem* P, double x, double xi) { return us_sample(P, x, xi); }
double orc_voigt(const orc_problem* P, double x) { return voigt_lookup(P, x); }
double orc_rkernel(const orc_problem* P, double D, double x, double g) { return r_kernel(P, D, x, g); }
