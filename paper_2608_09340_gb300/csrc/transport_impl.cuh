// Monte Carlo photon-packet walk (Sec. 2.1-2.3 of the paper), one persistent
// kernel per run.
//
// Scheduling: a persistent grid (a few CTAs per SM). Each lane owns one
// packet in registers. Whenever enough lanes of a warp are idle, the warp
// takes a contiguous block of packet ids with ONE atomicAdd on a global work
// counter (ballot + popc + shuffle) and the idle lanes emit those packets;
// this is the server-worker scheme of Sec. 2.3.2 at warp granularity. After
// the counter runs out, lanes finish their own packets independently.
//
// Per iteration a lane advances its packet by one event in the current
// cell: with x_com = x_lab - n.V/b (Sec. 2.2.1) and alpha = alpha0
// H(a, x_com) (Sec. 2.1), it either scatters inside the cell (tau < alpha
// s_exit) or crosses the nearest face. A scattering draws u_par from the
// velocity sampler (Sec. 2.1.1), u_perp from a Gaussian, an isotropic new
// direction and x_out = x_in + u_par (g - 1) + u_perp sin(gamma)
// (Eq. riia-scatter); with probability epsilon (Eq. eps) the photon is
// destroyed instead. Leaving a non-periodic face is an escape, binned in the
// lab-frame spectrum.
//
// Random numbers: Philox4x32-10 with counter (id_lo, id_hi, event, block)
// and key (seed_lo, seed_hi); a 32-bit word r becomes ((r >> 9) + 1/2) 2^-23,
// exact in FP32 and FP64. Event 0 is the emission, event e >= 1 the e-th
// scattering; the slots of each event are fixed (see emit / scatter), so a
// packet's stream depends only on (seed, id).
//
// Tallies: scattering counts and excitation are summed in registers over a
// cell visit and flushed with one atomic when the packet leaves the cell;
// the mean-intensity and emissivity tallies (Eq. scat-line) are added per
// segment. Spectrum and counters go to FP64 / 64-bit integers.
//
// Precision: R = float is the production walk (FP32 arithmetic in cell-local
// coordinates, so positions keep 2^-24 of a cell width at any optical depth);
// R = double runs the same steps in FP64 for lockstep checks.
#pragma once

#include <math.h>
#include <stdint.h>

#include "krl_internal.cuh"

namespace krl {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Table placement PH = 4 (a measurement variant of profile mode 2, chosen
// by krl_tune.table_space): the Voigt slice and the sampler's nodes and ln
// CDF read from __constant__ memory (60 KB, copied in before each launch)
// instead of shared memory; the search guides stay in shared memory. The
// arrays exist only in the translation unit that instantiates that mode.
#ifdef KRL_TABLES_IN_CONSTANT
__constant__ float c_voigt[kVoigtN];
__constant__ float c_usx[kUsNx];
__constant__ float c_uslncdf[kUsNx * kUsNu];
#endif

// ---------------------------------------------------------------- Philox4x32-10

struct Words {
    uint32_t w[4];
};

__device__ __forceinline__ Words philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const RoundKeys& K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t h0 = __umulhi(m0, c0), l0 = m0 * c0;
        uint32_t h1 = __umulhi(m1, c2), l1 = m1 * c2;
        uint32_t n0 = h1 ^ c1 ^ K.k[0][r];
        uint32_t n2 = h0 ^ c3 ^ K.k[1][r];
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
    }
    return Words{{c0, c1, c2, c3}};
}

// ---------------------------------------------------------------- precision policy

template <typename R>
struct Ops;

template <>
struct Ops<float> {
    // ((r >> 9) + 1/2) 2^-23 without an int-to-float conversion: the bits
    // give 1 + (r >> 9) 2^-23, and subtracting 1 - 2^-24 is exact (Sterbenz)
    static __device__ __forceinline__ float uni(uint32_t r)
    {
        return __uint_as_float((r >> 9) + 0x3f800000u) - 0x1.fffffep-1f;
    }
    static __device__ __forceinline__ float ln(float v) { return __logf(v); }
    static __device__ __forceinline__ float ex(float v) { return __expf(v); }
    // sqrt(v) for v >= 0 as v * rsqrt(v) (one MUFU op, 2 ulp)
    static __device__ __forceinline__ float sq(float v) { return v > 0.0f ? v * rsqrtf(v) : 0.0f; }
    static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
    // 1/a to about 1 ulp (one MUFU op; used for the exit distances only)
    static __device__ __forceinline__ float rcp(float a)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
    // sin and cos of 2 pi u for u in (0, 1): shift to [-pi, pi] where the
    // hardware approximation is accurate, then reflect.
    static __device__ __forceinline__ void sc2pi(float u, float* s, float* c)
    {
        float ss, cc;
        __sincosf(6.28318530717958648f * (u - 0.5f), &ss, &cc);
        *s = -ss;
        *c = -cc;
    }
    static __device__ __forceinline__ float big() { return 3.0e38f; }
    // min(1, max(0, p + d n)): one saturating FMA
    static __device__ __forceinline__ float step01(float p, float d, float n) { return __saturatef(fmaf(d, n, p)); }
    // position of |x| on the Voigt table, (log10|x| - L0) (N - 1) / (L1 - L0),
    // as one FMA on log2|x|
    static __device__ __forceinline__ float vt(float ax)
    {
        constexpr double C = (kVoigtN - 1) / (kVoigtL1 - kVoigtL0);
        return fmaf(__log2f(ax), (float)(C * 0.30102999566398119521), (float)(-kVoigtL0 * C));
    }
};

template <>
struct Ops<double> {
    static __device__ __forceinline__ double uni(uint32_t r) { return (double)(r >> 9) * 0x1p-23 + 0x1p-24; }
    static __device__ __forceinline__ double ln(double v) { return log(v); }
    static __device__ __forceinline__ double ex(double v) { return exp(v); }
    static __device__ __forceinline__ double sq(double v) { return sqrt(v); }
    static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
    static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
    static __device__ __forceinline__ void sc2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
    static __device__ __forceinline__ double big() { return 1.0e300; }
    static __device__ __forceinline__ double step01(double p, double d, double n) { return fmin(1.0, fmax(0.0, p + d * n)); }
    static __device__ __forceinline__ double vt(double ax)
    {
        return (log10(ax) - (double)kVoigtL0) * ((kVoigtN - 1) / (kVoigtL1 - kVoigtL0));
    }
};

// ---------------------------------------------------------------- paired FP32 draws
//
// The FP32 walk pairs the independent single-precision work of a scattering
// in the paired instructions of sm_100 and later (FFMA2 / FADD2 / FMUL2;
// each half rounds as the scalar operation would): the uniforms, the logs,
// the two angles, the square roots' products and the Box-Muller and
// direction products, and the two sampler rows' inversions.

__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a - b for two values as fma(b, -1, a): exact product, one rounding
__device__ __forceinline__ float2 sub2f(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

// two uniforms ((r >> 9) + 1/2) 2^-23, as Ops<float>::uni
__device__ __forceinline__ float2 uni2(uint32_t a, uint32_t b)
{
    return __fadd2_rn(make_float2(__uint_as_float((a >> 9) + 0x3f800000u), __uint_as_float((b >> 9) + 0x3f800000u)),
                      make_float2(-0x1.fffffep-1f, -0x1.fffffep-1f));
}

// One scattering's draws from its two Philox blocks (slots as in advance):
// the guide bin and L = ln(xi) of the velocity sampler, the Box-Muller
// radius and phase (cos, sin), the new isotropic direction, the next free
// path.
struct DrawsF {
    float L, rad, bc, bs, mx, my, mz, tau;
    int gm;
};

__device__ __forceinline__ DrawsF draws_f32(const Words& w0, const Words& w1)
{
    constexpr float kLn2 = 0.69314718055994531f;
    DrawsF D;
    const float2 ua = uni2(w0.w[0], w0.w[1]);          // xi of u_par, Box-Muller radius
    const float2 ub = uni2(w0.w[2], w0.w[3]);          // Box-Muller phase, free path
    const float2 uc = uni2(w1.w[0], w1.w[1]);          // mu, azimuth
    // -ln of the radius and free-path uniforms; ln xi and ln(1 - xi)
    const float2 nl = __fmul2_rn(make_float2(lg2_approx(ua.y), lg2_approx(ub.y)), make_float2(-kLn2, -kLn2));
    const float2 lx = __fmul2_rn(make_float2(lg2_approx(ua.x), lg2_approx(1.0f - ua.x)), make_float2(kLn2, kLn2));
    D.L = fminf(lx.x, -1e-30f);
    int m = (int)((D.L - lx.y + (float)kGuideW) * (float)(kGuideN / (2.0 * kGuideW)));
    D.gm = m < 0 ? 0 : (m > kGuideN - 1 ? kGuideN - 1 : m);
    D.tau = fmaxf(0.0f, nl.y);
    // square roots v rsqrt(v) of the radius^2 and of 1 - mu^2 (0 for v <= 0)
    const float rr = fmaxf(0.0f, nl.x);
    const float mu = fmaf(2.0f, uc.x, -1.0f);
    const float ss = fmaxf(0.0f, fmaf(-mu, mu, 1.0f));
    const float2 rt = __fmul2_rn(make_float2(rr, ss), make_float2(rsqrtf(rr), rsqrtf(ss)));
    D.rad = rr > 0.0f ? rt.x : 0.0f;
    const float st = ss > 0.0f ? rt.y : 0.0f;
    // sin and cos of 2 pi u through the shifted angle 2 pi (u - 1/2) in
    // [-pi, pi] (negated back), for the phase and the azimuth
    const float2 ang = __fmul2_rn(__fadd2_rn(make_float2(ub.x, uc.y), make_float2(-0.5f, -0.5f)),
                                  make_float2(6.28318530717958648f, 6.28318530717958648f));
    float sb, cb, sp, cp;
    __sincosf(ang.x, &sb, &cb);
    __sincosf(ang.y, &sp, &cp);
    D.bc = -cb;
    D.bs = -sb;
    const float2 mxy = __fmul2_rn(make_float2(st, st), make_float2(-cp, -sp));
    D.mx = mxy.x;
    D.my = mxy.y;
    D.mz = mu;
    return D;
}

// ---------------------------------------------------------------- table lookups (shared memory)

// H(a, x) from the ph_mode 2 slice: ln H linear in log10|x| between nodes;
// H(a, 0) below |x| = 1e-4 and the wing series above 1e3. The table path is
// evaluated for every x (finite for any x); the two outer ranges, which a
// walk rarely reaches, replace it in a branch of their own.
template <typename R>
__device__ __forceinline__ R voigt(R x, const float* sv, R a, R H0)
{
    using O = Ops<R>;
    const R ax = fabs(x);
    const R t = O::vt(ax);
    int i = (int)t;
    i = i < 0 ? 0 : (i > kVoigtN - 2 ? kVoigtN - 2 : i);
    const R f = t - (R)i;
    const R l0 = (R)sv[i], l1 = (R)sv[i + 1];
    R h = O::ex(((R)1 - f) * l0 + f * l1);
    if (ax < (R)1e-4 || ax > (R)1e3) {
        const R ax2 = ax * ax;
        R wing;
        if constexpr (sizeof(R) == 4) {
            const float r = Ops<float>::rcp(ax2);                 // one reciprocal: a r (1 + 3r/2) / sqrt(pi)
            wing = (a * 0.56418958354775628f) * r * fmaf(1.5f, r, 1.0f);
        } else {
            wing = a / ((R)1.7724538509055160 * ax2) * ((R)1 + (R)1.5 / ax2);
        }
        h = ax < (R)1e-4 ? H0 : wing;
    }
    return h;
}

// Line-profile mode 1: ln H bilinear in (log10 a, log10|x|) on the global
// two-dimensional table; the rows v2_row, v2_row + 1 and the weight v2_w of
// this a come with the launch. |x| below the first node takes the first
// node; the wing series above |x| = 1e3.
template <typename R>
__device__ __forceinline__ R voigt2d(const TransportArgs& A, R x, R a)
{
    using O = Ops<R>;
    const R ax = fabs(x);
    constexpr double C = (kV2Nx - 1) / (kVoigtL1 - kVoigtL0);
    R t;
    if constexpr (sizeof(R) == 4) {
        t = fmaf(__log2f(fmaxf(ax, 1e-4f)), (float)(C * 0.30102999566398119521), (float)(-kVoigtL0 * C));
    } else {
        t = (log10(ax < 1e-4 ? 1e-4 : ax) - kVoigtL0) * C;
    }
    t = t < (R)0 ? (R)0 : t;
    int i = (int)t;
    i = i > kV2Nx - 2 ? kV2Nx - 2 : i;
    const R f = t - (R)i;
    const float* r0 = A.voigt2d + (size_t)A.v2_row * kV2Nx;
    const float* r1 = r0 + kV2Nx;
    const R l0 = ((R)1 - f) * (R)__ldg(r0 + i) + f * (R)__ldg(r0 + i + 1);
    const R l1 = ((R)1 - f) * (R)__ldg(r1 + i) + f * (R)__ldg(r1 + i + 1);
    const R w = (R)A.v2_w;
    const R tab = O::ex(((R)1 - w) * l0 + w * l1);
    const R ax2 = ax * ax;
    const R wing = O::dv(a, (R)1.7724538509055160 * ax2) * ((R)1 + O::dv((R)1.5, ax2));
    return ax > (R)1e3 ? wing : tab;
}

// Line-profile mode 3: (1 - w) exp(-x^2) + w a / (sqrt(pi) (x^2 + a^2)) with
// w = [1 + tanh(2|x| - 2 u0)] / 2 = 1 / (1 + exp(4 (u0 - |x|))).
template <typename R>
__device__ __forceinline__ R blend(const TransportArgs& A, R x, R a)
{
    using O = Ops<R>;
    const R ax = fabs(x);
    const R w = O::dv((R)1, (R)1 + O::ex((R)4 * ((R)A.u0 - ax)));
    const R core = O::ex(-ax * ax);
    const R wing = O::dv(a, (R)1.7724538509055160 * (ax * ax + a * a));
    return ((R)1 - w) * core + w * wing;
}

template <typename R, int PH>
__device__ __forceinline__ R profile(const TransportArgs& A, R x, const float* sv, R a, R H0)
{
    // (PH 4 is mode 2 with its tables in constant memory: the slice below)
    if constexpr (PH == 1) return voigt2d<R>(A, x, a);
    else if constexpr (PH == 3) return blend<R>(A, x, a);
    else return voigt<R>(x, sv, a, H0);
}

// Largest row i in [0, 38] with X[i] <= ax, and the two bracketing nodes:
// the row guide's entry for the bin of ax (a node at or below ax), then one
// step up if the next node is also <= ax. The FP64 walk takes the bin of ax
// rounded toward zero, so the entry stays at or below ax there too.
template <typename R>
__device__ __forceinline__ int us_row2(R ax, const float* sx, const unsigned char* rg, R& x0, R& x1)
{
    float f;
    if constexpr (sizeof(R) == 4) f = ax;
    else f = __double2float_rz(ax);
    int t = (int)(__float_as_uint(f) >> 19) - (int)kRowGuideBase;
    t = t < 0 ? 0 : (t > kRowGuideN - 1 ? kRowGuideN - 1 : t);
    const int i = rg[t];
    const R g0 = (R)sx[i], g1 = (R)sx[i + 1];
    const R gp = (R)sx[i < kUsNx - 2 ? i + 2 : kUsNx - 1];
    const bool up = i < kUsNx - 2 && g1 <= ax;
    x0 = up ? g1 : g0;
    x1 = up ? gp : g1;
    return i + (up ? 1 : 0);
}

// u_par for incoming gas-frame frequency x (|x| <= 300), given L = ln(xi)
// and the guide bin m of logit(xi). Each bracketing row is inverted at L:
// the largest node j with c[j] <= L (the guide entry starts at or next to
// it; the bounded walks make the result exactly the bisection's), then u is
// linear between nodes j and j + 1; the two rows' u are interpolated in |x|.
// The two rows are walked together so their shared-memory loads overlap.
template <typename R>
__device__ __forceinline__ R us_sample(R x, R L, int m, const float* sx, const float* sc, const unsigned char* sg,
                                       const unsigned char* rg)
{
    using O = Ops<R>;
    const R ax = fabs(x);
    R x0, x1;
    const int i = us_row2(ax, sx, rg, x0, x1);
    const R t = O::dv(ax - x0, x1 - x0);
    const float* ra = sc + i * kUsNu;
    const float* rb = ra + kUsNu;
    int ja = sg[i * kGuideN + m];
    int jb = sg[(i + 1) * kGuideN + m];
    R a0 = (R)ra[ja], a1 = (R)ra[ja + 1];
    R b0 = (R)rb[jb], b1 = (R)rb[jb + 1];
    // Every row starts at the floor ln 1e-30 < L and ends at ln 1 = 0 > L
    // (L is the log of a uniform in [2^-24, 1 - 2^-24]), so both walks stop
    // inside the row without bound checks.
    for (;;) {
        const bool da = a0 > L;
        const bool db = b0 > L;
        if (!(da || db)) break;
        if (da) { --ja; a1 = a0; a0 = (R)ra[ja]; }
        if (db) { --jb; b1 = b0; b0 = (R)rb[jb]; }
    }
    for (;;) {
        const bool ua = a1 <= L;
        const bool ub = b1 <= L;
        if (!(ua || ub)) break;
        if (ua) { ++ja; a0 = a1; a1 = (R)ra[ja + 1]; }
        if (ub) { ++jb; b0 = b1; b1 = (R)rb[jb + 1]; }
    }
    R ua_, ub_;
    if constexpr (sizeof(R) == 4) {
        // both rows at once: u_j + du (L - c_j) / (c_j+1 - c_j)
        const float2 num = sub2f(make_float2(L, L), make_float2(a0, b0));
        const float2 den = sub2f(make_float2(a1, b1), make_float2(a0, b0));
        const float2 fr = __fmul2_rn(num, make_float2(O::rcp(den.x), O::rcp(den.y)));
        float2 u2 = __ffma2_rn(make_float2((float)kUsDu, (float)kUsDu), make_float2((float)ja, (float)jb),
                               make_float2((float)kUsU0, (float)kUsU0));
        u2 = __ffma2_rn(make_float2((float)kUsDu, (float)kUsDu), fr, u2);
        ua_ = u2.x;
        ub_ = u2.y;
    } else {
        ua_ = (R)kUsU0 + (R)kUsDu * (R)ja + (R)kUsDu * O::dv(L - a0, a1 - a0);
        ub_ = (R)kUsU0 + (R)kUsDu * (R)jb + (R)kUsDu * O::dv(L - b0, b1 - b0);
    }
    const R u = ((R)1 - t) * ua_ + t * ub_;
    return x < (R)0 ? -u : u;
}

// Guide bin of logit(xi) and L = ln(xi) (< 0 strictly: node 250, ln CDF = 0,
// always bounds the search).
template <typename R>
__device__ __forceinline__ int us_bin(R xi, R& L)
{
    using O = Ops<R>;
    L = fmin(O::ln(xi), (R)-1e-30);
    const R w = L - O::ln((R)1 - xi);
    int m = (int)((w + (R)kGuideW) * (R)(kGuideN / (2.0 * kGuideW)));
    return m < 0 ? 0 : (m > kGuideN - 1 ? kGuideN - 1 : m);
}

// ---------------------------------------------------------------- packet state

template <typename R>
struct Pkt {
    int cx, cy, cz, c;
    R px, py, pz;
    R nx, ny, nz;
    R ix, iy, iz;          // 1 / n
    R x, tau;
    float4 rec;            // current cell record
    uint32_t nscat, ncross, cell0;
    unsigned long long id;
    uint32_t vis_scat;     // scatterings in this cell visit
    R vis_exc;             // sum w ds H over this cell visit
    R wgt;                 // packet weight (continuum absorption; 1 otherwise)
    R vis_abs;             // weight absorbed by the continuum over this visit
    bool prev_scat;        // last event was a scattering (draw the next one early)
    uint32_t cellsum;      // FP64 walk: sum of the cells of its scatterings (mod 2^32)
};

// n . V/b of a cell, always evaluated in this one fixed order (explicit
// fused multiply-adds): the comoving frequency x_lab - n.V/b then recovers
// exactly the value that x_lab was built from (e.g. 0 for line-centre
// emission), whose sign the velocity sampler's symmetry depends on.
template <typename R>
__device__ __forceinline__ R vdot(R nx, R ny, R nz, const float4& rec)
{
    return fma(nz, (R)rec.w, fma(ny, (R)rec.z, nx * (R)rec.y));
}

// The FP64 walk keeps 1 / n with the direction (its face distances are
// taken every event, as the oracle takes them); the FP32 walk forms them
// only when a packet crosses a face.
template <typename R>
__device__ __forceinline__ void set_dir(Pkt<R>& p, R nx, R ny, R nz)
{
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    if constexpr (sizeof(R) == 8) {
        p.ix = Ops<R>::rcp(nx);
        p.iy = Ops<R>::rcp(ny);
        p.iz = Ops<R>::rcp(nz);
    }
}

// Distance (in cell widths) to the face ahead along one axis, from the
// in-cell coordinate q in [0, 1] and the direction component n with 1/n.
template <typename R>
__device__ __forceinline__ R face_dist(R q, R n, R in)
{
    if constexpr (sizeof(R) == 4) {
        return fmaf(-q, in, in > 0.0f ? in : 0.0f);      // (1 - q)/n or -q/n
    } else {
        return n > 0.0 ? (1.0 - q) * in : (n < 0.0 ? -q * in : 1.0e300);
    }
}

template <typename R>
__device__ __forceinline__ void iso_dir(R umu, R uphi, R& nx, R& ny, R& nz)
{
    R mu = (R)2 * umu - (R)1;
    R st = Ops<R>::sq(fmax((R)0, (R)1 - mu * mu));
    R s, c;
    Ops<R>::sc2pi(uphi, &s, &c);
    nx = st * c;
    ny = st * s;
    nz = mu;
}

__device__ __forceinline__ void spectrum_add(const TransportArgs& A, double x, double w)
{
    int b;
    if (x < A.spec_lo) b = 0;
    else if (x >= A.spec_hi) b = A.spec_n + 1;
    else {
        b = 1 + (int)floor((x - A.spec_lo) / (A.spec_hi - A.spec_lo) * A.spec_n);
        if (b > A.spec_n) b = A.spec_n;
    }
    atomicAdd(A.spec_w + b, w);
    atomicAdd(A.spec_c + b, 1ull);
}

template <typename R>
__device__ __forceinline__ void write_record(const TransportArgs& A, const Pkt<R>& p, uint16_t status)
{
    if (!A.rec) return;
    krl_packet_record r;
    r.x = (float)p.x;
    r.nscat = p.nscat;
    r.ncross = p.ncross;
    r.status = status;
    r.pad = 0;
    r.cell0 = p.cell0;
    r.scat_cells = sizeof(R) == 8 ? p.cellsum : 0u;
    A.rec[p.id - A.first] = r;
}

// Emission (event 0). Slots: block 0 = {mu, phi, tau, freq1},
// block 1 = {freq2, pos_a, pos_b, pos_c}, block 2 = {cell_hi, cell_lo}.
// Returns false if the source point lies outside the domain (the packet
// then leaves at once).
template <typename R, unsigned F>
__device__ bool emit(const TransportArgs& A, const RoundKeys& K, Pkt<R>& p)
{
    using O = Ops<R>;
    const uint32_t lo = (uint32_t)p.id, hi = (uint32_t)(p.id >> 32);
    Words b0 = philox(lo, hi, 0u, 0u, K);
    const bool need1 = A.src_kind != KRL_SRC_POINT || A.src_profile == KRL_PROFILE_GAUSSIAN;
    Words b1 = {{0u, 0u, 0u, 0u}};
    if (need1) b1 = philox(lo, hi, 0u, 1u, K);
    const int dims[3] = {A.nx, A.ny, A.nz};
    double X[3];
    R n[3];
    if (A.src_kind == KRL_SRC_BEAM) {
        n[0] = n[1] = n[2] = (R)0;
        n[A.src_axis] = (R)1;
        double pos[2] = {(double)O::uni(b1.w[1]), (double)O::uni(b1.w[2])};
        int q = 0;
        for (int d = 0; d < 3; ++d) {
            if (d == A.src_axis) { X[d] = 0.0; continue; }
            X[d] = (d == A.band_axis) ? A.band_lo + (A.band_hi - A.band_lo) * pos[q] : dims[d] * pos[q];
            ++q;
        }
    } else {
        iso_dir<R>(O::uni(b0.w[0]), O::uni(b0.w[1]), n[0], n[1], n[2]);
        if (A.src_kind == KRL_SRC_POINT) {
            X[0] = A.src_pos[0];
            X[1] = A.src_pos[1];
            X[2] = A.src_pos[2];
        } else if (A.src_kind == KRL_SRC_PLANE) {
            int q = 1;
            for (int d = 0; d < 3; ++d)
                X[d] = (d == A.src_axis) ? A.src_plane : dims[d] * (double)O::uni(b1.w[q++]);
        } else {
            Words b2 = philox(lo, hi, 0u, 2u, K);
            double uc = (double)(b2.w[0] >> 8) * 0x1p-24 + (double)(b2.w[1] >> 8) * 0x1p-48 + 0x1p-49;
            int l = 0, h = A.ncell - 1;              // first cell with cdf > uc
            while (l < h) {
                int m = (l + h) >> 1;
                if (A.src_cdf[m] > uc) h = m;
                else l = m + 1;
            }
            int cz = l / (A.nx * A.ny);
            int cy = (l / A.nx) % A.ny;
            int cx = l % A.nx;
            X[0] = cx + (double)O::uni(b1.w[1]);
            X[1] = cy + (double)O::uni(b1.w[2]);
            X[2] = cz + (double)O::uni(b1.w[3]);
        }
    }
    set_dir(p, n[0], n[1], n[2]);
    int ci[3];
    R pp[3];
    bool inside = true;
    for (int d = 0; d < 3; ++d) {
        double f = floor(X[d]);
        int c = (int)f;
        double q = X[d] - f;
        if (q == 0.0 && n[d] < (R)0) {
            c -= 1;
            q = 1.0;
        }
        if ((A.periodic >> d) & 1u) {
            c %= dims[d];
            if (c < 0) c += dims[d];
        }
        if (c < 0 || c >= dims[d]) inside = false;
        ci[d] = c;
        pp[d] = (R)q;
    }
    p.tau = fmax((R)0, -O::ln(O::uni(b0.w[2])));
    R xcom = (R)0;
    if (A.src_profile == KRL_PROFILE_GAUSSIAN) {
        R s, c;
        O::sc2pi(O::uni(b1.w[0]), &s, &c);
        xcom = O::sq(fmax((R)0, -O::ln(O::uni(b0.w[3])))) * c;
    }
    p.nscat = 0;
    p.ncross = 0;
    p.cellsum = 0;
    p.vis_scat = 0;
    p.vis_exc = (R)0;
    p.wgt = (R)1;
    p.vis_abs = (R)0;
    p.prev_scat = true;
    if (!inside) {
        p.x = xcom;
        p.cell0 = 0xFFFFFFFFu;
        return false;
    }
    p.cx = ci[0];
    p.cy = ci[1];
    p.cz = ci[2];
    p.px = pp[0];
    p.py = pp[1];
    p.pz = pp[2];
    p.c = (ci[2] * A.ny + ci[1]) * A.nx + ci[0];
    p.cell0 = (uint32_t)p.c;
    p.rec = __ldg(A.cells + p.c);
    R vdn = (F & F_VEL) ? vdot<R>(p.nx, p.ny, p.nz, p.rec) : (R)0;
    p.x = xcom + vdn;
    return true;
}

// Camera m's share of one segment's emissivity (Eq. scat-line with the
// trilinear R_IIA table, Eq. riia-table, or Eq. riia-inf for |x_in| >= 120):
// the channels k with |x_out,k - x_com| <= 10, x_out,k = -(x0 + (k + 1/2) dx)
// - n_cam.V/b, each receive base R(x_out,k - x_com; x_com, g), g = n.n_cam.
// emiss_setup holds what depends on the segment and camera only: the channel
// range, n_cam.V/b and either the table cell (g node kg, x node j, packed as
// kg << 8 | j, and the four (g, x) corner weights) or, in the wing limit
// (cell < 0), the Gaussian's normalisation (w00) and 1 / (2 var) (w01).
template <typename R>
struct EmSetup {
    int k0, k1;            // channel range; empty when k0 > k1
    int cell;              // kg << 8 | j, or -1
    R vc, sgn;             // n_cam.V/b; sign of x_com (R(D; -x, g) = R(-D; x, g))
    R w00, w01, w10, w11;
    R x0, dx;              // channel origin and width in x units
};

template <typename R, bool VEL>
__device__ __forceinline__ EmSetup<R> emiss_setup(const TransportArgs& A, int m, const float4& rec, R nx, R ny, R nz,
                                                  R xcom)
{
    EmSetup<R> S;
    S.x0 = (R)A.ch_x0;
    S.dx = (R)A.ch_dx;
    const R axc = fabs(xcom);
    S.sgn = xcom < (R)0 ? (R)-1 : (R)1;
    const R cx = (R)A.cam[m][0], cy = (R)A.cam[m][1], cz = (R)A.cam[m][2];
    R g = nx * cx + ny * cy + nz * cz;
    g = fmin((R)1, fmax((R)-1, g));
    S.vc = VEL ? vdot<R>(cx, cy, cz, rec) : (R)0;
    // channels with |x_out,k - x_com| <= 10
    const R ctr = Ops<R>::dv(-S.x0 - S.vc - xcom, S.dx) - (R)0.5;
    const R span = Ops<R>::dv((R)kRdMax, S.dx);
    const int k0 = (int)ceil(ctr - span) - 1;
    const int k1 = (int)floor(ctr + span) + 1;
    S.k0 = k0 < 0 ? 0 : k0;
    S.k1 = k1 > A.n_ch - 1 ? A.n_ch - 1 : k1;
    if (axc >= (R)kRxMax) {
        const R v = fmax((R)1 - g, (R)(kRsMin * kRsMin));
        S.cell = -1;
        S.w00 = (R)1 / Ops<R>::sq((R)6.283185307179586 * v);
        S.w01 = (R)0.5 / v;
        S.w10 = S.w11 = (R)0;
        return S;
    }
    const R fx = axc * (R)((kRnX - 1) / kRxMax);
    const R fg = (g + (R)1) * (R)((kRnG - 1) / 2.0);
    int j = (int)fx;
    int kg = (int)fg;
    j = j > kRnX - 2 ? kRnX - 2 : j;
    kg = kg > kRnG - 2 ? kRnG - 2 : kg;
    const R wx = fx - (R)j, wg = fg - (R)kg;
    S.cell = kg << 8 | j;
    S.w00 = ((R)1 - wg) * ((R)1 - wx);
    S.w01 = ((R)1 - wg) * wx;
    S.w10 = wg * ((R)1 - wx);
    S.w11 = wg * wx;
    return S;
}

// Channel k (kf = k as R) of a segment's camera share, added to out[k] (the
// cell's row of that camera's cube). QUAD reads the table regrouped by
// interpolation cell (two float4 loads), else the plain table (eight loads);
// the values and their order of combination are the same.
template <typename R, bool QUAD>
__device__ __forceinline__ void emiss_channel(const TransportArgs& A, float* out, const EmSetup<R>& S, R xcom, R base,
                                              int k, R kf)
{
    const R xo = -(S.x0 + (kf + (R)0.5) * S.dx) - S.vc;
    const R D = xo - xcom;
    if (fabs(D) > (R)kRdMax) return;
    if (S.cell < 0) {
        atomicAdd(out + k, (float)(base * S.w00 * Ops<R>::ex(-D * D * S.w01)));
        return;
    }
    const R Dd = S.sgn * D;
    const R fd = (Dd + (R)kRdMax) * (R)(1.0 / kRdStep);
    int i;
    R wd;
    if constexpr (sizeof(R) == 4) {
        // floor(fd) for 0 <= fd < 2^23 by a round-down add of 2^23 (exact),
        // clamped to the last interval, without float/int conversions
        const float t = __fadd_rd(fd, 8388608.0f) - 8388608.0f;
        const float fi = fminf(fmaxf(t, 0.0f), (float)(kRnD - 2));
        i = __float_as_int(fi + 8388608.0f) - 0x4B000000;
        wd = fd - fi;
    } else {
        i = (int)floor(fd);
        i = i < 0 ? 0 : (i > kRnD - 2 ? kRnD - 2 : i);
        wd = fd - (R)i;
    }
    const int kg = S.cell >> 8, j = S.cell & 255;
    R a0, a1;
    if constexpr (QUAD) {
        const float4* q = A.rquad + ((size_t)kg * (kRnX - 1) + j) * kRnD + i;
        const float4 q0 = __ldg(q), q1 = __ldg(q + 1);
        a0 = S.w00 * (R)q0.x + S.w01 * (R)q0.y + S.w10 * (R)q0.z + S.w11 * (R)q0.w;
        a1 = S.w00 * (R)q1.x + S.w01 * (R)q1.y + S.w10 * (R)q1.z + S.w11 * (R)q1.w;
    } else {
        const float* r00 = A.rtab + ((size_t)kg * kRnX + j) * kRnD;
        const float* r01 = r00 + kRnD;
        const float* r10 = r00 + (size_t)kRnX * kRnD;
        const float* r11 = r10 + kRnD;
        a0 = S.w00 * (R)__ldg(r00 + i) + S.w01 * (R)__ldg(r01 + i) + S.w10 * (R)__ldg(r10 + i) +
             S.w11 * (R)__ldg(r11 + i);
        a1 = S.w00 * (R)__ldg(r00 + i + 1) + S.w01 * (R)__ldg(r01 + i + 1) + S.w10 * (R)__ldg(r10 + i + 1) +
             S.w11 * (R)__ldg(r11 + i + 1);
    }
    const R val = ((R)1 - wd) * a0 + wd * a1;
    atomicAdd(out + k, (float)(base * val));
}

// Camera m's share deposited by one thread (inside the walk).
template <typename R, bool VEL>
__device__ __forceinline__ void emiss_camera(const TransportArgs& A, int m, int c, const float4& rec, R nx, R ny,
                                             R nz, R xcom, R base)
{
    const EmSetup<R> S = emiss_setup<R, VEL>(A, m, rec, nx, ny, nz, xcom);
    if (S.k0 > S.k1) return;
    float* out = A.emiss + ((size_t)m * A.ncell + c) * A.n_ch;
    R kf = (R)S.k0;
    for (int k = S.k0; k <= S.k1; ++k, kf += (R)1) emiss_channel<R, false>(A, out, S, xcom, base, k, kf);
}

// First stage of the two-stage emissivity deposit (FP32 walk): the segment
// (cell, base weight, x_com, direction) goes to the run's segment buffer,
// one slot range per converged group of lanes (one atomic on the buffer's
// counter). Returns false when the buffer is full; the caller then deposits
// the segment itself.
__device__ __forceinline__ bool append_segment(const TransportArgs& A, int c, float base, float xcom, float nx,
                                               float ny, float nz)
{
    const unsigned mask = __activemask();
    const unsigned lane = threadIdx.x & 31u;
    const int leader = __ffs(mask) - 1;
    unsigned long long first = 0;
    if ((int)lane == leader) first = atomicAdd(A.seg_count, (unsigned long long)__popc(mask));
    first = __shfl_sync(mask, first, leader);
    const unsigned long long i = first + __popc(mask & ((1u << lane) - 1u));
    if (i >= A.seg_cap) return false;
    A.seg[2 * i] = make_float4(__int_as_float(c), base, xcom, nx);
    A.seg[2 * i + 1] = make_float4(ny, nz, 0.0f, 0.0f);
    return true;
}

// Per-segment tallies of the rich mode: mean intensity by comoving channel
// and the camera-directed emissivity (Eq. scat-line). With a segment buffer
// (FP32 walk) the emissivity is deposited by the second stage instead.
template <typename R, unsigned F>
__device__ void rich_segment(const TransportArgs& A, const Pkt<R>& p, R ds, R xcom, R H, R w)
{
    if ((A.rich & KRL_TALLY_J) && A.n_ch > 0) {
        R q = Ops<R>::dv(-xcom - (R)A.ch_x0, (R)A.ch_dx);
        if (q >= (R)0 && q < (R)A.n_ch) atomicAdd(A.J + (size_t)p.c * A.n_ch + (int)q, (double)(w * ds));
    }
    if (!(A.rich & KRL_TALLY_EMISS) || A.n_ch <= 0) return;
    const R base = w * ds * (R)p.rec.x * H * (R)0.079577471545947668;   // 1 / 4 pi
    if constexpr (sizeof(R) == 4) {
        if (A.seg && append_segment(A, p.c, base, xcom, p.nx, p.ny, p.nz)) return;
    }
    for (int m = 0; m < A.n_cam; ++m)
        emiss_camera<R, (F & F_VEL) != 0>(A, m, p.c, p.rec, p.nx, p.ny, p.nz, xcom, base);
}

// Second stage of the emissivity deposit. A warp takes 32 consecutive
// segment records (one per lane, coalesced); per camera each lane works out
// its own segment's setup, then the warp deposits the segments one after the
// other with the setup broadcast from its lane and the lanes spread over the
// channel range, so that a segment's R_IIA reads fall on four table rows
// shared by the warp and its atomic additions on consecutive channels of one
// cell. The record count is read on the device (no host round trip between
// the stages).
constexpr int kDepositBlock = 256;

template <bool VEL>
__global__ void __launch_bounds__(kDepositBlock) k_emiss_deposit(const __grid_constant__ TransportArgs A)
{
    const unsigned long long cnt = *A.seg_count;
    const unsigned long long n = cnt < A.seg_cap ? cnt : A.seg_cap;
    const int lane = (int)(threadIdx.x & 31u);
    const unsigned long long stride = ((unsigned long long)gridDim.x * blockDim.x) & ~31ull;
    for (unsigned long long w = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ull; w < n;
         w += stride) {
        const unsigned long long i = w + (unsigned long long)lane;
        const bool valid = i < n;
        float4 r0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), r1 = r0;
        if (valid) {
            r0 = __ldg(A.seg + 2 * i);
            r1 = __ldg(A.seg + 2 * i + 1);
        }
        const int c = valid ? __float_as_int(r0.x) : 0;
        const float4 rec = (VEL && valid) ? __ldg(A.cells + c) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float base = r0.y, xcom = r0.z;
        for (int m = 0; m < A.n_cam; ++m) {
            const EmSetup<float> S = emiss_setup<float, VEL>(A, m, rec, r0.w, r1.x, r1.y, xcom);
            unsigned todo = __ballot_sync(kFull, valid && S.k0 <= S.k1);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1u;
                EmSetup<float> T;
                T.k0 = __shfl_sync(kFull, S.k0, src);
                T.k1 = __shfl_sync(kFull, S.k1, src);
                T.cell = __shfl_sync(kFull, S.cell, src);
                T.x0 = S.x0;
                T.dx = S.dx;
                T.vc = __shfl_sync(kFull, S.vc, src);
                T.sgn = __shfl_sync(kFull, S.sgn, src);
                T.w00 = __shfl_sync(kFull, S.w00, src);
                T.w01 = __shfl_sync(kFull, S.w01, src);
                T.w10 = __shfl_sync(kFull, S.w10, src);
                T.w11 = __shfl_sync(kFull, S.w11, src);
                const float xs = __shfl_sync(kFull, xcom, src);
                const float bs = __shfl_sync(kFull, base, src);
                const int cs = __shfl_sync(kFull, c, src);
                float* out = A.emiss + ((size_t)m * A.ncell + cs) * A.n_ch;
                float kf = (float)(T.k0 + lane);
                for (int k = T.k0 + lane; k <= T.k1; k += 32, kf += 32.0f)
                    emiss_channel<float, true>(A, out, T, xs, bs, k, kf);
            }
        }
    }
}

template <typename R, unsigned F>
__device__ __forceinline__ void flush_visit(const TransportArgs& A, Pkt<R>& p)
{
    if constexpr (sizeof(R) == 8) p.cellsum += p.vis_scat * (uint32_t)p.c;
    if ((F & F_SCAT) && p.vis_scat && A.scat) atomicAdd(A.scat + p.c, (unsigned long long)p.vis_scat);
    if ((F & F_RICH) && (A.rich & KRL_TALLY_EXC) && p.vis_exc != (R)0) atomicAdd(A.exc + p.c, (double)p.vis_exc);
    if ((F & F_RICH) && A.tau_abs && p.vis_abs != (R)0) atomicAdd(A.absw + p.c, (double)p.vis_abs);
    p.vis_scat = 0;
    p.vis_exc = (R)0;
    p.vis_abs = (R)0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Launch shape per instantiation: the lean FP32 walk runs 512-thread CTAs,
// two per SM (64 registers each); the FP64 and rich-tally walks need more
// registers and run 256-thread CTAs.
template <typename R, unsigned F>
constexpr int max_block() { return (sizeof(R) == 4 && !(F & F_RICH)) ? 512 : 256; }

// Per-lane event counters (summed over the CTA at the end of a model).
struct LaneStats {
    unsigned long long emit, esc, des, stuck, scat, cross, absorbed;
};

// ---------------------------------------------------------------- tail compaction
//
// Dynamic shared memory after the tables: a control block (the CTA's "ids
// ran out" flag and per-warp packet counts, double-buffered by round) and a
// stash that holds one packet per thread, field-major (one 32-bit word per
// field and slot, so consecutive slots fall in consecutive banks).
constexpr size_t kCtlOff = (kSmemBytes + 15) / 16 * 16;
constexpr int kCtlInts = 4 + 2 * 32;
constexpr size_t kStashOff = kCtlOff + (size_t)kCtlInts * sizeof(int);
// Events a lane runs between two compaction checks in the tail.
constexpr int kTailRound = 32;
// Bulk-phase iterations between two reads of the CTA's stop flag by a warp
// with no idle lane.
constexpr int kBulkCheck = 16;

// Words per stashed packet: cell (c, cx, cy, cz), nscat, ncross, cell0, id
// (2 words), the scattering-cell sum (FP64 walk), and px, py, pz, nx, ny, nz,
// x, tau (and the weight in the rich walk) in R.
template <typename R, unsigned F>
constexpr int stash_words() { return 9 + (sizeof(R) == 8 ? 1 : 0) + ((F & F_RICH) ? 9 : 8) * (int)(sizeof(R) / 4); }

template <typename R, unsigned F>
constexpr size_t smem_bytes(int block) { return kStashOff + (size_t)stash_words<R, F>() * 4u * (size_t)block; }

template <typename R>
__device__ __forceinline__ void put_r(uint32_t* w, int& f, int n, int slot, R v)
{
    if constexpr (sizeof(R) == 4) {
        w[(f++) * n + slot] = __float_as_uint(v);
    } else {
        w[(f++) * n + slot] = (uint32_t)__double2loint(v);
        w[(f++) * n + slot] = (uint32_t)__double2hiint(v);
    }
}

template <typename R>
__device__ __forceinline__ R get_r(const uint32_t* w, int& f, int n, int slot)
{
    if constexpr (sizeof(R) == 4) {
        return __uint_as_float(w[(f++) * n + slot]);
    } else {
        const uint32_t lo = w[(f++) * n + slot];
        const uint32_t hi = w[(f++) * n + slot];
        return __hiloint2double((int)hi, (int)lo);
    }
}

// Moves a packet into / out of stash slot `slot`. The visit tallies are
// flushed before (they belong to the cell visit, not the packet), and the
// derived fields (1/n, the cell record) are recomputed from the stored ones
// by the same functions, so a restored packet continues bit for bit as it
// would have in its old lane.
template <typename R, unsigned F>
__device__ __forceinline__ void stash_put(uint32_t* w, int n, int slot, const Pkt<R>& p)
{
    int f = 0;
    w[(f++) * n + slot] = (uint32_t)p.c;
    w[(f++) * n + slot] = (uint32_t)p.cx;
    w[(f++) * n + slot] = (uint32_t)p.cy;
    w[(f++) * n + slot] = (uint32_t)p.cz;
    w[(f++) * n + slot] = p.nscat;
    w[(f++) * n + slot] = p.ncross;
    w[(f++) * n + slot] = p.cell0;
    w[(f++) * n + slot] = (uint32_t)p.id;
    w[(f++) * n + slot] = (uint32_t)(p.id >> 32);
    if constexpr (sizeof(R) == 8) w[(f++) * n + slot] = p.cellsum;
    put_r<R>(w, f, n, slot, p.px);
    put_r<R>(w, f, n, slot, p.py);
    put_r<R>(w, f, n, slot, p.pz);
    put_r<R>(w, f, n, slot, p.nx);
    put_r<R>(w, f, n, slot, p.ny);
    put_r<R>(w, f, n, slot, p.nz);
    put_r<R>(w, f, n, slot, p.x);
    put_r<R>(w, f, n, slot, p.tau);
    if (F & F_RICH) put_r<R>(w, f, n, slot, p.wgt);
}

template <typename R, unsigned F>
__device__ __forceinline__ void stash_get(const TransportArgs& A, const uint32_t* w, int n, int slot, Pkt<R>& p)
{
    int f = 0;
    p.c = (int)w[(f++) * n + slot];
    p.cx = (int)w[(f++) * n + slot];
    p.cy = (int)w[(f++) * n + slot];
    p.cz = (int)w[(f++) * n + slot];
    p.nscat = w[(f++) * n + slot];
    p.ncross = w[(f++) * n + slot];
    p.cell0 = w[(f++) * n + slot];
    const uint32_t lo = w[(f++) * n + slot];
    const uint32_t hi = w[(f++) * n + slot];
    p.id = ((unsigned long long)hi << 32) | lo;
    if constexpr (sizeof(R) == 8) p.cellsum = w[(f++) * n + slot];
    p.px = get_r<R>(w, f, n, slot);
    p.py = get_r<R>(w, f, n, slot);
    p.pz = get_r<R>(w, f, n, slot);
    const R nx = get_r<R>(w, f, n, slot);
    const R ny = get_r<R>(w, f, n, slot);
    const R nz = get_r<R>(w, f, n, slot);
    set_dir(p, nx, ny, nz);
    p.x = get_r<R>(w, f, n, slot);
    p.tau = get_r<R>(w, f, n, slot);
    p.wgt = (F & F_RICH) ? get_r<R>(w, f, n, slot) : (R)1;
    p.rec = __ldg(A.cells + p.c);
    p.vis_scat = 0;
    p.vis_exc = (R)0;
    p.vis_abs = (R)0;
    p.prev_scat = true;
}

// ---------------------------------------------------------------- one event

// Continuum absorption over a segment of optical depth dt (Eq. scat-line):
// ab = 1 - exp(-dt) is the absorbed fraction of the weight, and the
// returned factor (1 - exp(-dt))/dt the segment's mean weight per unit
// starting weight (its series below dt = 1e-4).
template <typename R>
__device__ __forceinline__ R seg_factor(R dt, R& ab)
{
    if constexpr (sizeof(R) == 4) ab = -expm1f(-dt);
    else ab = -expm1(-dt);
    if (dt < (R)1e-4) return (R)1 - dt * ((R)0.5 - dt * ((R)(1.0 / 6.0) - dt * (R)(1.0 / 24.0)));
    return ab / dt;
}

// Advances an active packet by one event in its current cell (a scattering
// inside the cell or a crossing of the nearest face). Returns false when the
// packet has ended (escape, destruction or event budget).
template <typename R, unsigned F, int PH>
__device__ __forceinline__ bool advance(const TransportArgs& A, const RoundKeys& K, Pkt<R>& p, const float* sv,
                                        const float* sx, const float* sc, const unsigned char* sg,
                                        const unsigned char* rg, R a, R H0, LaneStats& st)
{
    using O = Ops<R>;
    if (p.nscat + p.ncross >= A.max_iters32) {
        flush_visit<R, F>(A, p);
        ++st.stuck;
        st.scat += p.nscat;
        st.cross += p.ncross;
        write_record(A, p, 3);
        return false;
    }
    // Draw the next scattering's random numbers up front, for every lane of
    // the converged group, when any of them last scattered (the common case
    // deep in the line core): the lanes then share one pass through Philox
    // instead of the few lanes that follow a face crossing drawing again in
    // a divergent branch, and the chains overlap the lookup's latency. A
    // lane whose event turns out to be a crossing discards its draw.
    const uint32_t idlo = (uint32_t)p.id, idhi = (uint32_t)(p.id >> 32);
    Words w0 = {{0u, 0u, 0u, 0u}}, w1 = {{0u, 0u, 0u, 0u}};
    const bool spec = __any_sync(__activemask(), p.prev_scat);
    if (spec) {
        w0 = philox(idlo, idhi, p.nscat + 1u, 0u, K);
        w1 = philox(idlo, idhi, p.nscat + 1u, 1u, K);
    }
    const R vdn = (F & F_VEL) ? vdot<R>(p.nx, p.ny, p.nz, p.rec) : (R)0;
    const R xcom = p.x - vdn;
    const R H = profile<R, PH>(A, xcom, sv, a, H0);
    const R alpha = (R)p.rec.x * H;
    bool scat;
    R ds, sx_ = (R)0, nd = (R)0;
    int axis = 0;
    if constexpr (sizeof(R) == 4) {
        // FP32: the packet scatters in this cell iff the point at distance
        // tau / alpha along n lies inside the cell ([0, 1] on every axis; a
        // line-free cell gives an infinite or NaN distance: outside). The
        // face distances are needed only for a crossing.
        ds = O::dv(p.tau, alpha);
        const float2 qxy = __ffma2_rn(make_float2(ds, ds), make_float2(p.nx, p.ny), make_float2(p.px, p.py));
        const float qz = fmaf(ds, p.nz, p.pz);
        const float2 hxy = __fadd2_rn(qxy, make_float2(-0.5f, -0.5f));
        scat = fabsf(hxy.x) <= 0.5f && fabsf(hxy.y) <= 0.5f && fabsf(qz - 0.5f) <= 0.5f;
        if (scat) {
            p.px = qxy.x;
            p.py = qxy.y;
            p.pz = qz;
        } else {
            // a zero component counts as +1e-30 (the packet then crosses that
            // face only from exactly on it), so that 1/n is finite and its
            // sign alone selects the face ahead
            const float ix = O::rcp(p.nx != 0.0f ? p.nx : 1e-30f);
            const float iy = O::rcp(p.ny != 0.0f ? p.ny : 1e-30f);
            const float iz = O::rcp(p.nz != 0.0f ? p.nz : 1e-30f);
            sx_ = face_dist<R>(p.px, p.nx, ix);
            nd = ix;
            const R ty = face_dist<R>(p.py, p.ny, iy);
            const R tz = face_dist<R>(p.pz, p.nz, iz);
            if (ty < sx_) { sx_ = ty; axis = 1; nd = iy; }
            if (tz < sx_) { sx_ = tz; axis = 2; nd = iz; }
            ds = sx_;
            p.px = O::step01(p.px, ds, p.nx);
            p.py = O::step01(p.py, ds, p.ny);
            p.pz = O::step01(p.pz, ds, p.nz);
        }
    } else {
        // FP64 (the lockstep walk): nearest face first, as the oracle does
        const R tx = face_dist<R>(p.px, p.nx, p.ix);
        const R ty = face_dist<R>(p.py, p.ny, p.iy);
        const R tz = face_dist<R>(p.pz, p.nz, p.iz);
        sx_ = tx;
        nd = p.ix;
        if (ty < sx_) { sx_ = ty; axis = 1; nd = p.iy; }
        if (tz < sx_) { sx_ = tz; axis = 2; nd = p.iz; }
        scat = p.tau < alpha * sx_;
        ds = scat ? O::dv(p.tau, alpha) : sx_;
        p.px = O::step01(p.px, ds, p.nx);
        p.py = O::step01(p.py, ds, p.ny);
        p.pz = O::step01(p.pz, ds, p.nz);
    }
    if (F & F_RICH) {
        // segment tallies at the mean weight along the segment; the weight
        // then decays by the continuum's absorption over it
        R wseg = p.wgt, ab = (R)0;
        if (A.tau_abs) wseg = p.wgt * seg_factor<R>((R)__ldg(A.tau_abs + p.c) * ds, ab);
        if (A.rich & KRL_TALLY_EXC) p.vis_exc += wseg * ds * H;
        if (A.rich & (KRL_TALLY_J | KRL_TALLY_EMISS)) rich_segment<R, F>(A, p, ds, xcom, H, wseg);
        if (A.tau_abs) {
            p.vis_abs += p.wgt * ab;
            p.wgt = p.wgt * ((R)1 - ab);
            if (p.wgt < (R)kWeightCut) {
                flush_visit<R, F>(A, p);
                ++st.absorbed;
                st.scat += p.nscat;
                st.cross += p.ncross;
                write_record(A, p, 4);
                return false;
            }
        }
    }
    p.prev_scat = scat;
    if (scat) {
        // ---- scattering (event e = nscat): block 0 = {u_par, bm_r, bm_phi, tau},
        //      block 1 = {mu, phi, eps_test, -}
        ++p.nscat;
        ++p.vis_scat;
        if (!spec) {
            w0 = philox(idlo, idhi, p.nscat, 0u, K);
            w1 = philox(idlo, idhi, p.nscat, 1u, K);
        }
        if ((F & F_RICH) && (A.rich & kRichEps)) {
            if (O::uni(w1.w[2]) < (R)__ldg(A.eps + p.c)) {
                flush_visit<R, F>(A, p);
                ++st.des;
                st.scat += p.nscat;
                st.cross += p.ncross;
                write_record(A, p, 2);
                return false;
            }
        }
        // independent long-latency work first: Box-Muller, new direction,
        // the sampler's logs; then the table walk
        R bs, bc, rad, mx, my, mz, L, tau_new, z1, z2;
        int gm;
        if constexpr (sizeof(R) == 4) {
            const DrawsF D = draws_f32(w0, w1);
            bs = D.bs;
            bc = D.bc;
            rad = D.rad;
            mx = D.mx;
            my = D.my;
            mz = D.mz;
            L = D.L;
            gm = D.gm;
            tau_new = D.tau;
            const float2 z = __fmul2_rn(make_float2(rad, rad), make_float2(bc, bs));
            z1 = z.x;
            z2 = z.y;
        } else {
            O::sc2pi(O::uni(w0.w[2]), &bs, &bc);
            rad = O::sq(fmax((R)0, -O::ln(O::uni(w0.w[1]))));
            iso_dir<R>(O::uni(w1.w[0]), O::uni(w1.w[1]), mx, my, mz);
            gm = us_bin<R>(O::uni(w0.w[0]), L);
            tau_new = fmax((R)0, -O::ln(O::uni(w0.w[3])));
            z1 = rad * bc;
            z2 = rad * bs;
        }
        const R us = us_sample<R>(xcom, L, gm, sx, sc, sg, rg);   // finite for any x; unused beyond 300
        const R upar = fabs(xcom) > (R)300 ? z2 : us;
        const R g = p.nx * mx + p.ny * my + p.nz * mz;
        const R sg_ = O::sq(fmax((R)0, (R)1 - g * g));
        const R xout = xcom + upar * (g - (R)1) + z1 * sg_;
        set_dir(p, mx, my, mz);
        const R vdo = (F & F_VEL) ? vdot<R>(mx, my, mz, p.rec) : (R)0;
        p.x = xout + vdo;
        p.tau = tau_new;
        return true;
    }
    // ---- cross the face on `axis`
    if constexpr (sizeof(R) == 4) p.tau = fmaxf(0.0f, p.tau - alpha * sx_);   // (the two tests may part at a tie)
    else p.tau -= alpha * sx_;
    ++p.ncross;
    flush_visit<R, F>(A, p);
    const int dim = axis == 0 ? A.nx : (axis == 1 ? A.ny : A.nz);
    const int stride = axis == 0 ? 1 : (axis == 1 ? A.nx : A.nx * A.ny);
    const int cur = axis == 0 ? p.cx : (axis == 1 ? p.cy : p.cz);
    // side from the sign of 1/n, which selected the face
    const int step = nd > (R)0 ? 1 : -1;
    int nc = cur + step;
    int dc = step * stride;
    const R pnew = step > 0 ? (R)0 : (R)1;
    if (axis == 0) p.px = pnew;
    else if (axis == 1) p.py = pnew;
    else p.pz = pnew;
    if (nc < 0 || nc >= dim) {
        if (!((A.periodic >> axis) & 1u)) {
            spectrum_add(A, (double)p.x, (double)p.wgt);
            ++st.esc;
            st.scat += p.nscat;
            st.cross += p.ncross;
            write_record(A, p, 1);
            return false;
        }
        if (nc < 0) { nc += dim; dc += dim * stride; }
        else { nc -= dim; dc -= dim * stride; }
    }
    if (axis == 0) p.cx = nc;
    else if (axis == 1) p.cy = nc;
    else p.cz = nc;
    p.c += dc;
    p.rec = __ldg(A.cells + p.c);
    return true;
}

// One model's walk by the whole CTA: stage the model's tables in shared
// memory, run packets until the model's id counter is exhausted and every
// lane has finished, then add the counters. Every thread of the CTA calls it.
//
// Bulk phase: each lane owns a packet; a warp refills its idle lanes with one
// atomic on the id counter (ballot + popc + shuffle). The first warp of the
// CTA that finds the counter exhausted raises a CTA flag, and every warp
// leaves the bulk phase at its next iteration.
//
// Tail phase (the remaining, typically longest packets): rounds of
// kTailRound events per lane; after each round the CTA counts its running
// packets and, if they occupy more warps than they would fill, moves them
// (through the shared-memory stash) to the lowest threads. Emptied warps
// then wait at the round barrier without issuing, so the surviving packets
// run in full warps instead of sharing the issue slots with idle lanes.
//
// Line-profile mode PH (2: the slice; 1: the global 2-D table, with the
// sampler also read from global memory; 3: the core-wing blend) selects the
// profile and where the sampler's tables are read from.
template <typename R, unsigned F, int PH>
__device__ __forceinline__ void run_model(const TransportArgs& A, const RoundKeys& K, float* sm)
{
    int* ctl = reinterpret_cast<int*>(reinterpret_cast<char*>(sm) + kCtlOff);
    uint32_t* stash = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(sm) + kStashOff);
    unsigned char* sgw = reinterpret_cast<unsigned char*>(sm + kSmemFloats);
    if constexpr (PH == 2) {
        for (int i = threadIdx.x; i < kVoigtN; i += blockDim.x) sm[kSmemVoigt + i] = A.voigt_lnH[i];
    }
    if constexpr (PH == 2 || PH == 3) {
        for (int i = threadIdx.x; i < kUsNx; i += blockDim.x) sm[kSmemUsX + i] = A.us_x[i];
        for (int i = threadIdx.x; i < kUsNx * kUsNu; i += blockDim.x) sm[kSmemUsC + i] = A.us_lncdf[i];
    }
    if constexpr (PH != 1) {
        for (int i = threadIdx.x; i < kUsNx * kGuideN; i += blockDim.x) sgw[i] = A.us_guide[i];
    }
    if (threadIdx.x == 0) ctl[0] = 0;
    __syncthreads();
    const float* sv = sm + kSmemVoigt;
    const float* sx = PH == 1 ? A.us_x : sm + kSmemUsX;
    const float* sc = PH == 1 ? A.us_lncdf : sm + kSmemUsC;
#ifdef KRL_TABLES_IN_CONSTANT
    if constexpr (PH == 4) {
        sv = c_voigt;
        sx = c_usx;
        sc = c_uslncdf;
    }
#endif
    const unsigned char* sg = PH == 1 ? A.us_guide : sgw;
    // the sampler's row guide, from the staged nodes (all profile modes)
    unsigned char* rgw = reinterpret_cast<unsigned char*>(sm) + kSmemRowGuide;
    for (int t = threadIdx.x; t < kRowGuideN; t += blockDim.x) {
        const float edge = __uint_as_float((unsigned)(t + (int)kRowGuideBase) << 19);
        int i = 0;
        while (i < kUsNx - 2 && sx[i + 1] <= edge) ++i;
        rgw[t] = (unsigned char)i;
    }
    __syncthreads();
    const unsigned char* rg = rgw;

    const R a = (R)A.a;
    const R H0 = (R)__ldg(A.H0);
    const unsigned lane = threadIdx.x & 31u;
    const int warp = (int)(threadIdx.x >> 5);
    const int nwarps = (int)(blockDim.x >> 5);
    Pkt<R> p;
    bool active = false;
    LaneStats st = {0, 0, 0, 0, 0, 0, 0};

    // Both phases run in one loop so that the event code is inlined once.
    const int n = (int)blockDim.x;
    bool bulk = true;
    int round = 0, it = 0, quiet = 0;
    for (;;) {
        // ---- bulk phase: refill idle lanes, leave when the ids run out. A
        // warp whose lanes are all busy skips this bookkeeping, except every
        // kBulkCheck-th iteration, when it looks at the CTA's stop flag (the
        // other warps may be waiting for it at the tail barrier).
        const unsigned idle = bulk ? __ballot_sync(kFull, !active) : 0u;
        if (bulk && (idle != 0u || ++quiet == kBulkCheck)) {
            quiet = 0;
            const int nidle = __popc(idle);
            // lane 0 reads the flag and broadcasts it: every lane of the warp
            // must take the same decision (the leave path has a CTA barrier),
            // and lanes that read it themselves could see it before and after
            // another warp's write
            int stop = 0;
            if (lane == 0) stop = *reinterpret_cast<volatile int*>(ctl);
            bool leave = __shfl_sync(kFull, stop, 0) != 0;
            if (!leave && (nidle == 32 || (nidle > 0 && nidle >= A.refill_min))) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(A.next, (unsigned long long)nidle);
                base = __shfl_sync(kFull, base, 0);
                leave = base + (unsigned long long)nidle >= A.n;
                if (leave && lane == 0) *reinterpret_cast<volatile int*>(ctl) = 1;
                if (!active) {
                    const unsigned long long k = base + __popc(idle & ((1u << lane) - 1u));
                    if (k < A.n) {
                        p.id = A.first + k;
                        ++st.emit;
                        if (emit<R, F>(A, K, p)) {
                            active = true;
                        } else {
                            spectrum_add(A, (double)p.x, 1.0);
                            ++st.esc;
                            write_record(A, p, 1);
                        }
                    }
                }
            }
            if (leave) {                      // warp-uniform; once per warp
                bulk = false;
                __syncthreads();
            }
        } else if (!bulk && (it == kTailRound || !__any_sync(kFull, active))) {
            // ---- tail phase, end of a round: count and compact
            const unsigned m = __ballot_sync(kFull, active);
            int* cnt = ctl + 4 + 32 * (round & 1);
            if (lane == 0) cnt[warp] = __popc(m);
            __syncthreads();
            int total = 0, before = 0, busy = 0;
            for (int w = 0; w < nwarps; ++w) {
                const int c = cnt[w];
                total += c;
                before += w < warp ? c : 0;
                busy += c > 0 ? 1 : 0;
            }
            if (total == 0) break;            // CTA-uniform
            if (busy > (total + 31) / 32) {   // CTA-uniform
                if (active) {
                    flush_visit<R, F>(A, p);
                    stash_put<R, F>(stash, n, before + __popc(m & ((1u << lane) - 1u)), p);
                }
                __syncthreads();
                // the stash is next written after a later round's count
                // barrier, which every thread reaches only after this read
                active = (int)threadIdx.x < total;
                if (active) stash_get<R, F>(A, stash, n, (int)threadIdx.x, p);
            }
            ++round;
            it = 0;
        }
        if (!bulk) ++it;
        if (active) active = advance<R, F, PH>(A, K, p, sv, sx, sc, sg, rg, a, H0, st);
    }

    const unsigned long long tot[7] = {warp_sum(st.emit),  warp_sum(st.esc),  warp_sum(st.des),
                                       warp_sum(st.stuck), warp_sum(st.scat), warp_sum(st.cross),
                                       warp_sum(st.absorbed)};
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 7; ++k)
            if (tot[k]) atomicAdd(A.stats + k, tot[k]);
    }
}

template <typename R, unsigned F, int PH>
__global__ void __launch_bounds__(max_block<R, F>(), 2) k_transport(const __grid_constant__ TransportArgs A)
{
    extern __shared__ float sm[];
    run_model<R, F, PH>(A, A.keys, sm);
}

// The lowest-numbered model that still has unassigned packet ids, or -1.
// The shared cursor only moves forward, so the loop ends within n_models
// steps.
__device__ int next_model(const BatchArgs& B)
{
    int m = atomicAdd(B.cursor, 0);
    while (m < B.n_models) {
        const unsigned long long used = atomicAdd(B.models[m].next, 0ull);
        if (used < B.models[m].n) return m;
        atomicCAS(B.cursor, m, m + 1);
        const int m2 = atomicAdd(B.cursor, 0);
        m = m2 > m ? m2 : m + 1;
    }
    return -1;
}

// Many independent models (grids) in one persistent launch: each CTA takes
// the lowest model that still has packets, stages that model's tables,
// runs its warps on it until its ids run out, drains, and takes the next.
// CTAs finish models at different times, so one model's tail overlaps the
// next model's bulk instead of idling the device as separate launches do.
// The batched launch runs 256-thread CTAs (smaller CTAs move on to the next
// model sooner; the autotuner found them faster on uneven model sets).
constexpr int kBatchBlock = 256;

template <typename R, unsigned F>
__global__ void __launch_bounds__(kBatchBlock, 2) k_transport_batch(const __grid_constant__ BatchArgs B)
{
    extern __shared__ float sm[];
    __shared__ TransportArgs sA;
    __shared__ int s_model;
    for (;;) {
        if (threadIdx.x == 0) s_model = next_model(B);
        __syncthreads();
        const int m = s_model;
        if (m < 0) break;
        {
            const int* src = reinterpret_cast<const int*>(B.models + m);
            int* dst = reinterpret_cast<int*>(&sA);
            for (int i = threadIdx.x; i < (int)(sizeof(TransportArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        run_model<R, F, 2>(sA, B.keys, sm);
        __syncthreads();     // every warp done before the tables are replaced
    }
}

template <typename R, unsigned F, int PH>
cudaError_t launch_one(const TransportArgs& A, int grid, int block, cudaStream_t s)
{
    if (block > max_block<R, F>()) return cudaErrorInvalidConfiguration;
    auto kern = k_transport<R, F, PH>;
    // the shared-memory opt-in is an attribute of the kernel on the current
    // device: set it on every launch (a host-side call of about a
    // microsecond), so that a launch on any device of the process has it
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes<R, F>(max_block<R, F>()));
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem_bytes<R, F>(block), s>>>(A);
    return cudaGetLastError();
}

template <typename R, unsigned F>
cudaError_t launch_batch_one(const BatchArgs& B, int grid, int block, cudaStream_t s)
{
    if (block > kBatchBlock) return cudaErrorInvalidConfiguration;
    auto kern = k_transport_batch<R, F>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes<R, F>(kBatchBlock));   // per device: every launch
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem_bytes<R, F>(block), s>>>(B);
    return cudaGetLastError();
}

template <typename R, unsigned F, int PH>
int occupancy_one(int block)
{
    if (block > max_block<R, F>()) return 0;
    auto kern = k_transport<R, F, PH>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<R, F>(max_block<R, F>()));
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, smem_bytes<R, F>(block)) != cudaSuccess) return 0;
    return n;
}

template <typename R, int PH>
cudaError_t dispatch(const TransportArgs& A, unsigned f, int grid, int block, cudaStream_t s)
{
    switch (f & 7u) {
    case 0: return launch_one<R, 0, PH>(A, grid, block, s);
    case 1: return launch_one<R, 1, PH>(A, grid, block, s);
    case 2: return launch_one<R, 2, PH>(A, grid, block, s);
    case 3: return launch_one<R, 3, PH>(A, grid, block, s);
    case 4: return launch_one<R, 4, PH>(A, grid, block, s);
    case 5: return launch_one<R, 5, PH>(A, grid, block, s);
    case 6: return launch_one<R, 6, PH>(A, grid, block, s);
    default: return launch_one<R, 7, PH>(A, grid, block, s);
    }
}

template <typename R, unsigned F>
int batch_occupancy_one(int block)
{
    if (block > kBatchBlock) return 0;
    auto kern = k_transport_batch<R, F>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<R, F>(kBatchBlock));
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, smem_bytes<R, F>(block)) != cudaSuccess) return 0;
    return n;
}

template <typename R>
int batch_occ_dispatch(unsigned f, int block)
{
    switch (f & 7u) {
    case 0: return batch_occupancy_one<R, 0>(block);
    case 1: return batch_occupancy_one<R, 1>(block);
    case 2: return batch_occupancy_one<R, 2>(block);
    case 3: return batch_occupancy_one<R, 3>(block);
    case 4: return batch_occupancy_one<R, 4>(block);
    case 5: return batch_occupancy_one<R, 5>(block);
    case 6: return batch_occupancy_one<R, 6>(block);
    default: return batch_occupancy_one<R, 7>(block);
    }
}

template <typename R>
cudaError_t dispatch_batch(const BatchArgs& B, unsigned f, int grid, int block, cudaStream_t s)
{
    switch (f & 7u) {
    case 0: return launch_batch_one<R, 0>(B, grid, block, s);
    case 1: return launch_batch_one<R, 1>(B, grid, block, s);
    case 2: return launch_batch_one<R, 2>(B, grid, block, s);
    case 3: return launch_batch_one<R, 3>(B, grid, block, s);
    case 4: return launch_batch_one<R, 4>(B, grid, block, s);
    case 5: return launch_batch_one<R, 5>(B, grid, block, s);
    case 6: return launch_batch_one<R, 6>(B, grid, block, s);
    default: return launch_batch_one<R, 7>(B, grid, block, s);
    }
}

template <typename R, int PH>
int occ_dispatch(unsigned f, int block)
{
    switch (f & 7u) {
    case 0: return occupancy_one<R, 0, PH>(block);
    case 1: return occupancy_one<R, 1, PH>(block);
    case 2: return occupancy_one<R, 2, PH>(block);
    case 3: return occupancy_one<R, 3, PH>(block);
    case 4: return occupancy_one<R, 4, PH>(block);
    case 5: return occupancy_one<R, 5, PH>(block);
    case 6: return occupancy_one<R, 6, PH>(block);
    default: return occupancy_one<R, 7, PH>(block);
    }
}

}  // namespace
}  // namespace krl
