// Deterministic channel-map ray trace (Sec. 2.2.2, Eq. imaging-formal and
// Eq. imaging-alphas): the second step of the two-step imaging scheme,
// turning the camera-directed emissivity of the Monte Carlo pass into
// velocity-channel maps.
//
// Orthographic camera: pixel-centred parallel rays along the camera
// direction n (image axes e_theta, e_phi of the camera angles), centred on
// the box. For a cell segment of length dl and channel k, with gas-frame
// frequency x_k = -(v_k + n.V)/b,
//   alpha_k = alpha0 H(a, x_k) + alpha_abs,  dtau = alpha_k dl,
//   I_out = I_in e^{-dtau} + j_k dl (1 - e^{-dtau}) / dtau,
//   j_k = j_sca,k + j_line H(a, x_k) / sqrt(pi),
// i.e. S_k = j_k / alpha_k in Eq. imaging-formal, finite for empty cells;
// alpha_abs is the continuum absorption (zero without one), applied here in
// the imaging pass as the two-step scheme does (Sec. 3.2).
//
// GPU layout: per camera, a prep kernel tabulates the channel extinction
// alpha_k per (cell, channel) (it depends on the cell and the channel only);
// the trace then gives each ray a group of lanes with the channels across
// them (4 per lane), so that a cell's [n_ch] rows are coalesced reads and a
// warp follows several neighbouring rays. Without memory for the cube, one
// warp per pixel evaluates the profile per segment. Rays are marched from
// the camera side backwards; each channel sums
// I = sum_seg T j dl f(dtau) with T = exp(-tau in front of the segment), the
// optical depth and the sum carried with compensated (Kahan) addition so
// that FP32 stays within 1e-5 of an FP64 trace over hundreds of segments.
#include <math.h>

#include "krl_internal.cuh"

namespace krl {

namespace {

// H(a, x) from the ph_mode 2 slice with the node position resolved to
// ~2e-5 of a node: |x| = m 2^e with e exact, t = IT_e + FT_e + C log10(m)
// where IT_e + FT_e = C (e log10 2 + 4) is precomputed (integer and
// fractional part) and C = 4999 / 7; a plain FP32 evaluation of t ~ 3000
// would keep only ~1e-4 of its fraction.
constexpr int kRtEmin = -16;
constexpr int kRtEn = 30;

__device__ __forceinline__ float voigt_rt(float x, const float* sv, const int* eI, const float* eF, float a,
                                          float H0)
{
    float ax = fabsf(x);
    if (ax < 1e-4f) return H0;
    if (ax > 1e3f) return a / (1.7724538509055160f * ax * ax) * (1.0f + 1.5f / (ax * ax));
    int e;
    float m = frexpf(ax, &e);                       // ax = m 2^e, m in [0.5, 1)
    int q = e - kRtEmin;
    q = q < 0 ? 0 : (q > kRtEn - 1 ? kRtEn - 1 : q);
    // C log10(m) = (C log10 2) log2(m); |log2 m| <= 1, so the fast log2's
    // absolute error (~2^-22) moves t by < 5e-5
    const float sfr = eF[q] + (float)((kVoigtN - 1) / (kVoigtL1 - kVoigtL0) * 0.30102999566398119521) * __log2f(m);
    const float fl = floorf(sfr);
    int i = eI[q] + (int)fl;
    float f = sfr - fl;
    if (i < 0) { i = 0; f = 0.0f; }
    if (i > kVoigtN - 2) { i = kVoigtN - 2; f = 1.0f; }
    return __expf((1.0f - f) * sv[i] + f * sv[i + 1]);
}

// (1 - e^{-d}) / d: from e^{-d} above d = 0.05 (cancellation below 1.2e-6),
// by its Taylor series below (truncation below 5e-10).
__device__ __forceinline__ float escape_factor(float d)
{
    if (d > 0.05f) return __fdividef(1.0f - __expf(-d), d);
    return 1.0f - d * (0.5f - d * (1.0f / 6.0f - d * (1.0f / 24.0f - d * (1.0f / 120.0f))));
}

// Error-free sum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// n . V with n given as float pairs (nh + nl) and V in float, returned as a
// float pair (hi, lo) accurate to ~1e-14 relative: products split exactly
// with FMA, partial sums carried with two_sum. Replaces an FP64 evaluation,
// whose rate on this part would dominate the walk.
__device__ __forceinline__ void dot_ff(const float* nh, const float* nl, float v0, float v1, float v2,
                                       float& hi, float& lo)
{
    const float v[3] = {v0, v1, v2};
    float s = 0.0f, c = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float p = nh[d] * v[d];
        const float pe = fmaf(nh[d], v[d], -p);
        float t, te;
        two_sum(s, p, t, te);
        s = t;
        c += te + pe + nl[d] * v[d];
    }
    hi = s + c;
    lo = c - (hi - s);
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v)
{
    float y = v - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Per-camera profile cube: for every (cell, channel), H(a, x_k) with
// x_k = -(v_k + n.V)/b, or (ALPHA) the extinction alpha0 H + alpha_abs. Along one camera direction x_k depends on the cell
// and the channel only, not on the ray, so the trace reads it from here
// instead of evaluating the profile for each of the ~16 rays that cross a
// cell. The arithmetic is the trace's own (float-pair n.V, exponent-split
// table index). One warp per cell, channels across lanes.
template <int CPL, bool ALPHA>
__global__ void __launch_bounds__(256) k_rt_profile(const RayArgs A, float* hc)
{
    __shared__ float sv[kVoigtN];
    __shared__ int eI[kRtEn];
    __shared__ float eF[kRtEn];
    for (int i = threadIdx.x; i < kVoigtN; i += blockDim.x) sv[i] = A.voigt_lnH[i];
    if (threadIdx.x < kRtEn) {
        const double t = (double)((kVoigtN - 1) / (kVoigtL1 - kVoigtL0)) *
                         (((int)threadIdx.x + kRtEmin) * 0.30102999566398119521 - kVoigtL0);
        const double it = floor(t);
        eI[threadIdx.x] = (int)it;
        eF[threadIdx.x] = (float)(t - it);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long ncell = (long long)A.nx * A.ny * A.nz;
    float nh[3], nl[3];
    for (int d = 0; d < 3; ++d) {
        nh[d] = (float)A.n[d];
        nl[d] = (float)(A.n[d] - (double)nh[d]);
    }
    float xbh[CPL], xbl[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const double xb = -(A.ch_x0 + ((double)(lane + 32 * q) + 0.5) * A.ch_dx);
        xbh[q] = (float)xb;
        xbl[q] = (float)(xb - (double)xbh[q]);
    }
    const float a = A.a;
    const float H0 = __ldg(A.H0);
    // a warp takes 32 consecutive cells: each lane forms one cell's n.V (and
    // reads its record), then the warp fills the cells' channel rows one
    // after the other with those values broadcast
    const long long ngroups = (ncell + 31) / 32;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long grp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; grp < ngroups; grp += nwarps) {
        const long long c0 = grp * 32;
        const long long cl = c0 + lane;
        float vnh = 0.0f, vnl = 0.0f, a0 = 0.0f, ta = 0.0f;
        if (cl < ncell) {
            const float4 rec = __ldg(A.cells + cl);
            a0 = rec.x;
            if (ALPHA && A.tau_abs) ta = __ldg(A.tau_abs + cl);
            dot_ff(nh, nl, rec.y, rec.z, rec.w, vnh, vnl);
        }
        const int cells = ncell - c0 < 32 ? (int)(ncell - c0) : 32;
        for (int i = 0; i < cells; ++i) {
            const float h = __shfl_sync(0xffffffffu, vnh, i), l = __shfl_sync(0xffffffffu, vnl, i);
            const float ca = __shfl_sync(0xffffffffu, a0, i), ct = __shfl_sync(0xffffffffu, ta, i);
            float* row = hc + (size_t)(c0 + i) * A.n_ch;
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const int k = lane + 32 * q;
                if (k < A.n_ch) {
                    const float xk = (xbh[q] - h) + (xbl[q] - l);
                    const float H = voigt_rt(xk, sv, eI, eF, a, H0);
                    row[k] = ALPHA ? fmaf(ca, H, ct) : H;
                }
            }
        }
    }
}

// Each ray's start on the camera-side face of the box, one thread per ray
// (FP64: the entry point fixes the segment lengths of the whole ray): the
// first cell and the position inside it, or no hit. The trace's lanes read
// their ray's record instead of repeating this setup per lane.
__global__ void __launch_bounds__(256) k_ray_setup(const RayArgs A)
{
    const long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long npix = (long long)A.npix_x * A.npix_y;
    if (ray >= npix) return;
    const int ix = (int)(ray % A.npix_x);
    const int iy = (int)(ray / A.npix_x);
    const double uc = (ix + 0.5) * A.pix - 0.5 * A.pix * A.npix_x;
    const double vc = (iy + 0.5) * A.pix - 0.5 * A.pix * A.npix_y;
    double P[3];
    for (int d = 0; d < 3; ++d) P[d] = A.centre[d] + uc * A.u[d] + vc * A.v[d];
    const double hi[3] = {(double)A.nx, (double)A.ny, (double)A.nz};
    double t0 = -1e300, t1 = 1e300;
    bool hit = true;
    for (int d = 0; d < 3; ++d) {
        if (A.n[d] != 0.0) {
            double ta = (0.0 - P[d]) / A.n[d], tb = (hi[d] - P[d]) / A.n[d];
            t0 = fmax(t0, fmin(ta, tb));
            t1 = fmin(t1, fmax(ta, tb));
        } else if (!(P[d] >= 0.0 && P[d] < hi[d])) {
            hit = false;
        }
    }
    hit = hit && t1 > t0;
    int ci[3] = {0, 0, 0};
    float p[3] = {0.0f, 0.0f, 0.0f};
    if (hit) {
        for (int d = 0; d < 3; ++d) {
            double X = fmin(hi[d], fmax(0.0, P[d] + t1 * A.n[d]));
            double f = floor(X);
            int c = (int)f;
            double r = X - f;
            const float dir = (float)(-A.n[d]);
            if (r == 0.0 && dir < 0.0f) { c -= 1; r = 1.0; }
            if (c >= (int)hi[d]) { c = (int)hi[d] - 1; r = 1.0; }
            ci[d] = c;
            p[d] = (float)r;
        }
    }
    A.rayinit[2 * ray] = make_float4(__int_as_float(ci[0]), __int_as_float(ci[1]), __int_as_float(ci[2]),
                                     __int_as_float(hit ? 1 : 0));
    A.rayinit[2 * ray + 1] = make_float4(p[0], p[1], p[2], 0.0f);
}

// Two channels at a time with the paired FP32 instructions (sm_100 and
// later; each half rounds as the single-precision operation would). a - b
// is formed as fma(b, -1, a), exact in the product and rounded once.
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

__device__ __forceinline__ void kahan_add2(float2& sum, float2& comp, float2 v)
{
    const float2 y = sub2(v, comp);
    const float2 t = __fadd2_rn(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
}

// e^{-x} of two values as 2^(-x log2 e), with the hardware's approximate
// base-2 exponential
__device__ __forceinline__ float2 exp_neg2(float2 x)
{
    const float2 m = __fmul2_rn(x, make_float2(-1.4426950408889634f, -1.4426950408889634f));
    float2 r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(m.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(m.y));
    return r;
}

// (1 - e^{-d})/d of two values without a branch: from e^{-d} above d = 0.05,
// else its Taylor series 1 - d/2 + d^2/6 - d^3/24 + d^4/120 (Horner in d)
__device__ __forceinline__ float2 escape_factor2(float2 d)
{
    const float2 e = exp_neg2(d);
    float2 rd;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd.x) : "f"(d.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd.y) : "f"(d.y));
    const float2 lg = __fmul2_rn(sub2(make_float2(1.0f, 1.0f), e), rd);
    float2 sm = __ffma2_rn(make_float2(1.0f / 120.0f, 1.0f / 120.0f), d, make_float2(-1.0f / 24.0f, -1.0f / 24.0f));
    sm = __ffma2_rn(sm, d, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
    sm = __ffma2_rn(sm, d, make_float2(-0.5f, -0.5f));
    sm = __ffma2_rn(sm, d, make_float2(1.0f, 1.0f));
    return make_float2(d.x > 0.05f ? lg.x : sm.x, d.y > 0.05f ? lg.y : sm.y);
}

// One cell's extinction and emissivity for a lane's four channels, as two
// pairs. FULL (n_ch = 4 LPR, rows 16-byte aligned): lane `sub` of a ray holds
// channels 4 sub .. 4 sub + 3, read as one 16-byte vector per row, so a
// ray's lanes read each row in one contiguous sweep. Otherwise pair h holds
// channels sub + LPR (2h) and sub + LPR (2h + 1); channels past n_ch read zeros
// (dtau = 0 and no intensity).
template <int LPR, bool FULL>
__device__ __forceinline__ void cell_rows(const RayArgs& A, int c, int sub, float2 (&v)[2], float2 (&j)[2])
{
    const float* arow = A.hcube + (size_t)c * A.n_ch;
    const float* jrow = A.emiss + (size_t)c * A.n_ch;
    if constexpr (FULL) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(arow) + sub);
        const float4 e = __ldg(reinterpret_cast<const float4*>(jrow) + sub);
        v[0] = make_float2(a.x, a.y);
        v[1] = make_float2(a.z, a.w);
        j[0] = make_float2(e.x, e.y);
        j[1] = make_float2(e.z, e.w);
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ka = sub + LPR * (2 * h), kb = ka + LPR;
            v[h] = make_float2(ka < A.n_ch ? __ldg(arow + ka) : 0.0f, kb < A.n_ch ? __ldg(arow + kb) : 0.0f);
            j[h] = make_float2(ka < A.n_ch ? __ldg(jrow + ka) : 0.0f, kb < A.n_ch ? __ldg(jrow + kb) : 0.0f);
        }
    }
}

// Channel of element e of pair h of lane `sub` (the layout of cell_rows).
template <int LPR, bool FULL>
__device__ __forceinline__ int lane_channel(int sub, int h, int e)
{
    return FULL ? 4 * sub + 2 * h + e : sub + LPR * (2 * h + e);
}

// The trace over the per-camera cube (k_rt_profile): LPR lanes per ray, 4
// channels per lane, so a warp follows 32 / LPR neighbouring rays, whose
// walks through the grid nearly coincide. The per-segment work (face
// distances, cell index) is shared by fewer lanes' worth of channels than
// with one ray per warp. The cube holds the extinction alpha0 H + alpha_abs
// (JL false) or H (JL true: the line-emission term needs H; alpha is formed
// here).
template <int LPR, bool JL, bool FULL>
__global__ void __launch_bounds__(256, 4) k_trace_cube(const RayArgs A)
{
    constexpr int CPL = 4;
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPR;
    const long long ray = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / LPR) + lane / LPR;
    const long long npix = (long long)A.npix_x * A.npix_y;
    if (ray >= npix) return;                 // no warp-wide operations follow
    const int ix = (int)(ray % A.npix_x);
    const int iy = (int)(ray / A.npix_x);

    // the ray's start (k_ray_setup): first cell, position in it, hit
    const float4 r0 = __ldg(A.rayinit + 2 * ray), r1 = __ldg(A.rayinit + 2 * ray + 1);
    // the lane's channel pairs: intensity, optical depth in front of the
    // segment, and their compensation terms
    float2 I[CPL / 2], Ic[CPL / 2], tau[CPL / 2], tc[CPL / 2];
#pragma unroll
    for (int h = 0; h < CPL / 2; ++h) I[h] = Ic[h] = tau[h] = tc[h] = make_float2(0.0f, 0.0f);

    if (__float_as_int(r0.w)) {
        // cell and in-cell position as scalars (an array indexed by the
        // crossing axis would live in local memory); the crossing axis is
        // applied by selects
        int ci0 = __float_as_int(r0.x), ci1 = __float_as_int(r0.y), ci2 = __float_as_int(r0.z);
        float p0 = r1.x, p1 = r1.y, p2 = r1.z;
        const float d0 = A.dirf[0], d1 = A.dirf[1], d2 = A.dirf[2];
        const int nx = A.nx, ny = A.ny, nz = A.nz, nxy = A.nx * A.ny;
        // the ray's start can lie outside (a ray along the box's face); after
        // that only the axis just stepped on can leave the box
        const bool inside = ci0 >= 0 && ci0 < nx && ci1 >= 0 && ci1 < ny && ci2 >= 0 && ci2 < nz;
        const unsigned fwd = (d0 > 0.0f ? 1u : 0u) | (d1 > 0.0f ? 2u : 0u) | (d2 > 0.0f ? 4u : 0u);
        const int max_seg = inside ? nx + ny + nz + 3 : 0;
        int c = (ci2 * ny + ci1) * nx + ci0;
        for (int seg = 0; seg < max_seg; ++seg) {
            // distance to the face ahead on each axis, one FMA each
            float s = fmaf(p0, A.face_neg[0], A.face_c[0]);
            int axis = 0;
            const float t1 = fmaf(p1, A.face_neg[1], A.face_c[1]);
            if (t1 < s) { s = t1; axis = 1; }
            const float t2 = fmaf(p2, A.face_neg[2], A.face_c[2]);
            if (t2 < s) { s = t2; axis = 2; }
            float2 v[2], j[2];
            cell_rows<LPR, FULL>(A, c, sub, v, j);
            float a0 = 0.0f, ta = 0.0f, jl = 0.0f;
            if (JL) {
                a0 = __ldg(A.cells + c).x;
                ta = A.tau_abs ? __ldg(A.tau_abs + c) : 0.0f;
                jl = __ldg(A.jline + c) * 0.56418958354775628f;
            }
            const float2 s2 = make_float2(s, s);
#pragma unroll
            for (int h = 0; h < CPL / 2; ++h) {
                float2 vv = v[h], jj = j[h];
                if (JL) {
                    jj = __ffma2_rn(make_float2(jl, jl), vv, jj);
                    vv = __ffma2_rn(make_float2(a0, a0), vv, make_float2(ta, ta));
                }
                const float2 dtau = __fmul2_rn(vv, s2);
                const float2 T = exp_neg2(tau[h]);
                kahan_add2(I[h], Ic[h], __fmul2_rn(__fmul2_rn(__fmul2_rn(T, jj), s2), escape_factor2(dtau)));
                kahan_add2(tau[h], tc[h], dtau);
            }
            // move to the face, then step across it (the crossing axis is set exactly)
            p0 = __saturatef(fmaf(s, d0, p0));
            p1 = __saturatef(fmaf(s, d1, p1));
            p2 = __saturatef(fmaf(s, d2, p2));
            const bool x0 = axis == 0, x1 = axis == 1;
            const bool up = (fwd >> axis) & 1u;
            const int nc = (x0 ? ci0 : (x1 ? ci1 : ci2)) + (up ? 1 : -1);
            const int dim = x0 ? nx : (x1 ? ny : nz);
            if ((unsigned)nc >= (unsigned)dim) break;
            const float pn = up ? 0.0f : 1.0f;
            ci0 = x0 ? nc : ci0;
            ci1 = x1 ? nc : ci1;
            ci2 = (x0 || x1) ? ci2 : nc;
            p0 = x0 ? pn : p0;
            p1 = x1 ? pn : p1;
            p2 = (x0 || x1) ? p2 : pn;
            const int stride = x0 ? 1 : (x1 ? nx : nxy);
            c += up ? stride : -stride;
        }
    }
#pragma unroll
    for (int h = 0; h < CPL / 2; ++h) {
        const int ka = lane_channel<LPR, FULL>(sub, h, 0), kb = lane_channel<LPR, FULL>(sub, h, 1);
        if (ka < A.n_ch) A.maps[((size_t)ka * A.npix_y + iy) * A.npix_x + ix] = I[h].x;
        if (kb < A.n_ch) A.maps[((size_t)kb * A.npix_y + iy) * A.npix_x + ix] = I[h].y;
    }
}

// Without the per-camera cube (its memory not available): one warp per
// pixel, the profile evaluated per segment.
template <int CPL>
__global__ void __launch_bounds__(256) k_raytrace(const RayArgs A)
{
    __shared__ float sv[kVoigtN];
    __shared__ int eI[kRtEn];
    __shared__ float eF[kRtEn];
    for (int i = threadIdx.x; i < kVoigtN; i += blockDim.x) sv[i] = A.voigt_lnH[i];
    if (threadIdx.x < kRtEn) {
        const double t = (double)((kVoigtN - 1) / (kVoigtL1 - kVoigtL0)) *
                         (((int)threadIdx.x + kRtEmin) * 0.30102999566398119521 - kVoigtL0);
        const double it = floor(t);
        eI[threadIdx.x] = (int)it;
        eF[threadIdx.x] = (float)(t - it);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long npix = (long long)A.npix_x * A.npix_y;
    if (warp >= npix) return;
    const int ix = (int)(warp % A.npix_x);
    const int iy = (int)(warp / A.npix_x);
    const float a = A.a;
    const float H0 = __ldg(A.H0);

    // ray setup in FP64: pixel centre on the image plane, box entry/exit
    const double uc = (ix + 0.5) * A.pix - 0.5 * A.pix * A.npix_x;
    const double vc = (iy + 0.5) * A.pix - 0.5 * A.pix * A.npix_y;
    double P[3], n[3];
    for (int d = 0; d < 3; ++d) {
        P[d] = A.centre[d] + uc * A.u[d] + vc * A.v[d];
        n[d] = A.n[d];
    }
    const double hi[3] = {(double)A.nx, (double)A.ny, (double)A.nz};
    double t0 = -1e300, t1 = 1e300;
    bool hit = true;
    for (int d = 0; d < 3; ++d) {
        if (n[d] != 0.0) {
            double ta = (0.0 - P[d]) / n[d], tb = (hi[d] - P[d]) / n[d];
            t0 = fmax(t0, fmin(ta, tb));
            t1 = fmin(t1, fmax(ta, tb));
        } else if (!(P[d] >= 0.0 && P[d] < hi[d])) {
            hit = false;
        }
    }
    float I[CPL], Ic[CPL], tau[CPL], tc[CPL], xbh[CPL], xbl[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        I[q] = Ic[q] = tau[q] = tc[q] = 0.0f;
        // -v_k / b as a float pair (hi + lo)
        const double xb = -(A.ch_x0 + ((double)(lane + 32 * q) + 0.5) * A.ch_dx);
        xbh[q] = (float)xb;
        xbl[q] = (float)(xb - (double)xbh[q]);
    }

    if (hit && t1 > t0) {
        // start on the camera-side face and march along -n
        int ci[3];
        float p[3], dir[3], inv[3];
        for (int d = 0; d < 3; ++d) {
            double X = fmin(hi[d], fmax(0.0, P[d] + t1 * n[d]));
            double f = floor(X);
            int c = (int)f;
            double r = X - f;
            dir[d] = (float)(-n[d]);
            if (r == 0.0 && dir[d] < 0.0f) { c -= 1; r = 1.0; }
            if (c >= (int)hi[d]) { c = (int)hi[d] - 1; r = 1.0; }
            ci[d] = c;
            p[d] = (float)r;
            inv[d] = 1.0f / dir[d];
        }
        float nh[3], nl[3];
        for (int d = 0; d < 3; ++d) {
            nh[d] = (float)n[d];
            nl[d] = (float)(n[d] - (double)nh[d]);
        }
        const int max_seg = A.nx + A.ny + A.nz + 3;
        for (int seg = 0; seg < max_seg; ++seg) {
            if (ci[0] < 0 || ci[0] >= A.nx || ci[1] < 0 || ci[1] >= A.ny || ci[2] < 0 || ci[2] >= A.nz) break;
            float s = 3.0e38f;
            int axis = 0;
            for (int d = 0; d < 3; ++d) {
                float t = dir[d] > 0.0f ? (1.0f - p[d]) * inv[d] : (dir[d] < 0.0f ? -p[d] * inv[d] : 3.0e38f);
                if (t < s) { s = t; axis = d; }
            }
            const int c = (ci[2] * A.ny + ci[1]) * A.nx + ci[0];
            const float4 rec = __ldg(A.cells + c);
            // n . V/b (|V/b| reaches tens) as a float pair
            float vnh, vnl;
            dot_ff(nh, nl, rec.y, rec.z, rec.w, vnh, vnl);
            const float jl = A.jline ? __ldg(A.jline + c) : 0.0f;
            const float ta = A.tau_abs ? __ldg(A.tau_abs + c) : 0.0f;
            const float* jrow = A.emiss + (size_t)c * A.n_ch;
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const int k = lane + 32 * q;
                if (k < A.n_ch) {
                    const float xk = (xbh[q] - vnh) + (xbl[q] - vnl);
                    const float H = voigt_rt(xk, sv, eI, eF, a, H0);
                    const float dtau = fmaf(rec.x, H, ta) * s;
                    float j = __ldg(jrow + k);
                    if (A.jline) j = fmaf(jl * 0.56418958354775628f, H, j);
                    const float T = __expf(-tau[q]);
                    kahan_add(I[q], Ic[q], T * j * s * escape_factor(dtau));
                    kahan_add(tau[q], tc[q], dtau);
                }
            }
            for (int d = 0; d < 3; ++d)
                if (d != axis) p[d] = fminf(1.0f, fmaxf(0.0f, fmaf(s, dir[d], p[d])));
            const int step = dir[axis] > 0.0f ? 1 : -1;
            ci[axis] += step;
            p[axis] = step > 0 ? 0.0f : 1.0f;
        }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int k = lane + 32 * q;
        if (k < A.n_ch) A.maps[((size_t)k * A.npix_y + iy) * A.npix_x + ix] = I[q];
    }
}

}  // namespace

// The profile cube (when A.hcube), then the trace over it with LPR lanes
// per ray; without the cube, the one-ray-per-warp trace that evaluates the
// profile per segment.
template <int CPL, int LPR>
cudaError_t launch_cpl(const RayArgs& A, int sm_count, cudaStream_t s)
{
    const long long npix = (long long)A.npix_x * A.npix_y;
    if (A.hcube) {
        const long long blocks = (npix * LPR + 255) / 256;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        k_ray_setup<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(A);
        // the vector reads need each lane's four channels 16-byte aligned
        const bool full = A.n_ch == 4 * LPR && (reinterpret_cast<uintptr_t>(A.emiss) & 15u) == 0 &&
                          (reinterpret_cast<uintptr_t>(A.hcube) & 15u) == 0;
        if (A.jline) {
            k_rt_profile<CPL, false><<<sm_count * 8, 256, 0, s>>>(A, A.hcube);
            if (full) k_trace_cube<LPR, true, true><<<(unsigned)blocks, 256, 0, s>>>(A);
            else k_trace_cube<LPR, true, false><<<(unsigned)blocks, 256, 0, s>>>(A);
        } else {
            k_rt_profile<CPL, true><<<sm_count * 8, 256, 0, s>>>(A, A.hcube);
            if (full) k_trace_cube<LPR, false, true><<<(unsigned)blocks, 256, 0, s>>>(A);
            else k_trace_cube<LPR, false, false><<<(unsigned)blocks, 256, 0, s>>>(A);
        }
    } else {
        const long long blocks = (npix * 32 + 255) / 256;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        k_raytrace<CPL><<<(unsigned)blocks, 256, 0, s>>>(A);
    }
    return cudaGetLastError();
}

cudaError_t launch_raytrace(const RayArgs& A, int sm_count, cudaStream_t s)
{
    if (A.n_ch <= 4) return launch_cpl<1, 1>(A, sm_count, s);
    if (A.n_ch <= 8) return launch_cpl<1, 2>(A, sm_count, s);
    if (A.n_ch <= 16) return launch_cpl<1, 4>(A, sm_count, s);
    if (A.n_ch <= 32) return launch_cpl<1, 8>(A, sm_count, s);
    if (A.n_ch <= 64) return launch_cpl<2, 16>(A, sm_count, s);
    if (A.n_ch <= 128) return launch_cpl<4, 32>(A, sm_count, s);
    return cudaErrorInvalidValue;
}

}  // namespace krl
