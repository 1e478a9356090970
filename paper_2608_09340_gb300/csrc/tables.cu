// Per-line setup on the device, all arithmetic in FP64, results stored as
// float32 (the method builds its tables in double precision and keeps them
// in single precision, Sec. 2.3):
//
//  * the ph_mode 2 Voigt slice H(a, |x|) at 5000 nodes uniform in log10|x|
//    on [-4, 3], stored as ln H (Sec. 2.2.1, 2.3.1);
//  * the velocity sampler (Sec. 2.1.1): 40 incoming-frequency rows (18
//    uniform below |x| = 8, 22 log-spaced to 300) of ln CDF of
//    p(u | x) ~ exp(-u^2) / (a^2 + (x-u)^2) at 251 u-nodes on [-6, 6];
//  * the R_IIA kernel table (Eq. riia-table) on 201 Delta x 200 |x| x 40 g
//    nodes, built from the same discrete sampler masses;
//  * per-cell records {line-centre tau per cell width, V/b} (Eq. sigma0),
//    destruction probabilities (Eq. eps) and the emission CDF over cells.
#include <math.h>

#include "krl_internal.cuh"
#include "voigt.cuh"

namespace krl {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Fourier coefficients of Weideman's expansion, one thread per coefficient.
__global__ void k_weideman(double* c, int N, double L)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (n > N) return;
    const int M = 2 * N;
    double s = 0.0;
    for (int k = -M + 1; k <= M - 1; ++k) {
        double th = k * kPi / M;
        double t = L * tan(0.5 * th);
        s += (L * L + t * t) * exp(-t * t) * cos(n * th);
    }
    c[n - 1] = s / (2.0 * M);
}

__global__ void k_voigt(double a, const double* c, int N, double L, float* lnH, float* H0)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kVoigtN) {
        double l = kVoigtL0 + (kVoigtL1 - kVoigtL0) * i / (kVoigtN - 1);
        double x = pow(10.0, l);
        lnH[i] = (float)log(voigt_H(a, x, c, N, L));
    }
    if (i == 0) *H0 = (float)voigt_H(a, 0.0, c, N, L);
}

// Line-profile mode 1 table: ln H(a_j, x_i) with log10 a_j uniform on
// [kV2LaMin, kV2LaMax] (kV2Na nodes) and log10 x_i uniform on [kVoigtL0,
// kVoigtL1] (kV2Nx nodes); one thread per entry.
__global__ void k_voigt2d(const double* c, int N, double L, float* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kV2Na * kV2Nx) return;
    const int j = k / kV2Nx, i = k % kV2Nx;
    const double a = pow(10.0, kV2LaMin + (kV2LaMax - kV2LaMin) * j / (kV2Na - 1));
    const double x = pow(10.0, kVoigtL0 + (kVoigtL1 - kVoigtL0) * i / (kV2Nx - 1));
    out[k] = (float)log(voigt_H(a, x, c, N, L));
}

// Mass of p(u | x) in the u-cell [lo, hi]: the Lorentz factor L(u) times
// the second-order expansion of exp(-u^2) about the midpoint m, integrated
// exactly: exp(-m^2) [I0 - 2 m I1 + (2 m^2 - 1) I2], Ik = int (u-m)^k L du.
// u-node j = -6 + 0.048 j, rounded after the product and after the sum (no
// fused multiply-add): the node at u = 0 must be exactly 0, because for a
// tiny damping parameter a shift of 1e-16 moves the Lorentz spike of width a
// across a cell edge.
__device__ __forceinline__ double unode(int j) { return __dadd_rn(kUsU0, __dmul_rn(kUsDu, (double)j)); }

__device__ double cell_mass(double x, double a, int j)
{
    double lo = unode(j);
    double hi = unode(j + 1);
    double m = 0.5 * (lo + hi);
    double dl = lo - x, dh = hi - x;
    // Lorentz integral (atan(dh/a) - atan(dl/a)) / a; when the cell lies on
    // one side of x the two angles nearly cancel for small a, so use
    // atan(A) - atan(B) = atan((A - B) / (1 + A B)) there
    double I0 = (dl * dh > 0.0) ? atan((hi - lo) * a / (a * a + dl * dh)) / a
                                : (atan(dh / a) - atan(dl / a)) / a;
    double Jx = 0.5 * log((a * a + dh * dh) / (a * a + dl * dl));
    double xm = x - m;
    double I1 = Jx + xm * I0;
    double I2 = (hi - lo) - a * a * I0 + 2.0 * xm * Jx + xm * xm * I0;
    return exp(-m * m) * (I0 - 2.0 * m * I1 + (2.0 * m * m - 1.0) * I2);
}

__device__ double us_xnode(int i)
{
    return i < 18 ? 8.0 * i / 18.0 : 8.0 * pow(37.5, (i - 18) / 21.0);
}

// One thread per sampler row: sequential cumulative sum, then ln CDF and
// the row's search guide.
// One block per row: the cell masses in parallel, then the normalisation
// and running sums by one thread in index order (the same sums, in the same
// order, as a serial build), the logs in parallel, the guide by one thread.
__global__ void k_usampler(double a, float* xs, float* lncdf, unsigned char* guide)
{
    __shared__ double mass[kUsNu - 1];
    __shared__ double cdf[kUsNu];
    const int i = blockIdx.x;
    const double x = us_xnode(i);
    for (int j = threadIdx.x; j < kUsNu - 1; j += blockDim.x) mass[j] = cell_mass(x, a, j);
    __syncthreads();
    if (threadIdx.x == 0) {
        xs[i] = (float)x;
        double tot = 0.0;
        for (int j = 0; j < kUsNu - 1; ++j) tot += mass[j];
        double run = 0.0;
        cdf[0] = 0.0;
        for (int j = 1; j < kUsNu; ++j) {
            run += mass[j - 1];
            cdf[j] = run / tot;
        }
    }
    __syncthreads();
    float* row = lncdf + (size_t)i * kUsNu;
    for (int j = threadIdx.x; j < kUsNu; j += blockDim.x) {
        const double C = cdf[j];
        row[j] = (float)log(j > 0 && C > kUsFloor ? C : kUsFloor);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned char* gd = guide + (size_t)i * kGuideN;
        int j = 0;
        for (int m = 0; m < kGuideN; ++m) {
            double w = -kGuideW + 2.0 * kGuideW * m / kGuideN;
            double lt = -log1p(exp(-w));          // ln sigmoid(w)
            while (j < kUsNu - 2 && (double)row[j + 1] <= lt) ++j;
            gd[m] = (unsigned char)j;
        }
    }
}

// Normalised sampler masses at the R-table |x| nodes: p[jx][k].
__global__ void k_rmasses(double a, double* p)
{
    int jx = blockIdx.x * blockDim.x + threadIdx.x;
    if (jx >= kRnX) return;
    double x = kRxMax * jx / (kRnX - 1);
    double* row = p + (size_t)jx * (kUsNu - 1);
    double tot = 0.0;
    for (int k = 0; k < kUsNu - 1; ++k) {
        double m = cell_mass(x, a, k);
        row[k] = m;
        tot += m;
    }
    for (int k = 0; k < kUsNu - 1; ++k) row[k] /= tot;
}

// rquad(k, j, i) = the R table's four (g, x) corners of cell (k, j) at Delta_i.
__global__ void k_rquad(const float* rtab, float4* rquad)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kRquadElems) return;
    const int i = (int)(e % kRnD);
    const int j = (int)((e / kRnD) % (kRnX - 1));
    const int k = (int)(e / ((size_t)kRnD * (kRnX - 1)));
    const float* r00 = rtab + ((size_t)k * kRnX + j) * kRnD + i;
    rquad[e] = make_float4(r00[0], r00[kRnD], r00[(size_t)kRnX * kRnD], r00[(size_t)kRnX * kRnD + kRnD]);
}

// R(D_i; x_j, g_k) = sum_c p_c G(D_i - m_c (g_k - 1); s_k), one thread per entry.
__global__ void k_rtable(const double* p, float* rtab)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kRtabElems) return;
    int i = (int)(e % kRnD);
    int jx = (int)((e / kRnD) % kRnX);
    int kg = (int)(e / ((size_t)kRnD * kRnX));
    double D = -kRdMax + kRdStep * i;
    double g = -1.0 + 2.0 * kg / (kRnG - 1);
    double sg = sqrt(fmax(0.0, 1.0 - g * g)) / sqrt(2.0);
    double s = sg > kRsMin ? sg : kRsMin;
    double inv2s2 = 0.5 / (s * s);
    double norm = 1.0 / (sqrt(2.0 * kPi) * s);
    const double* row = p + (size_t)jx * (kUsNu - 1);
    double acc = 0.0;
    for (int c = 0; c < kUsNu - 1; ++c) {
        double lo = unode(c);
        double hi = unode(c + 1);
        double m = 0.5 * (lo + hi);
        double y = D - m * (g - 1.0);
        acc += row[c] * exp(-y * y * inv2s2);
    }
    rtab[e] = (float)(acc * norm);
}

__global__ void k_fields(FieldArgs F)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= F.ncell) return;
    double tau = (double)F.opacity[c] * F.tau_scale;
    float4 r;
    r.x = (float)tau;
    r.y = F.vx ? (float)((double)F.vx[c] * F.inv_b) : 0.0f;
    r.z = F.vy ? (float)((double)F.vy[c] * F.inv_b) : 0.0f;
    r.w = F.vz ? (float)((double)F.vz[c] * F.inv_b) : 0.0f;
    F.cells[c] = r;
    if (F.eps) {
        double q = F.n_coll ? F.k_ul * (double)F.n_coll[c] : 0.0;
        F.eps[c] = (float)(q / (F.A_ul + q));
    }
}

__global__ void k_validate(const float* f, int n, int allow_negative, int* bad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = f[i];
    if (!isfinite(v) || (!allow_negative && v < 0.0f)) atomicOr(bad, 1);
}

// Block-level inclusive scan in FP64, 256 threads x 8 elements per block.
constexpr int kScanT = 256;
constexpr int kScanE = 8;
constexpr int kScanChunk = kScanT * kScanE;

__device__ double block_inclusive_scan(double v, double* sh)
{
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < kScanT; off <<= 1) {
        double add = t >= off ? sh[t - off] : 0.0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    double r = sh[t];
    __syncthreads();
    return r;
}

__global__ void k_scan_local(const float* rate, int n, double* out, double* block_tot, int* bad)
{
    __shared__ double sh[kScanT];
    size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanE;
    double v[kScanE];
    double run = 0.0;
    for (int e = 0; e < kScanE; ++e) {
        size_t i = base + e;
        double r = 0.0;
        if (i < (size_t)n) {
            float f = rate[i];
            if (!isfinite(f) || f < 0.0f) atomicOr(bad, 1);
            r = (double)f;
        }
        run += r;
        v[e] = run;
    }
    double incl = block_inclusive_scan(run, sh);
    double excl = incl - run;
    for (int e = 0; e < kScanE; ++e) {
        size_t i = base + e;
        if (i < (size_t)n) out[i] = v[e] + excl;
    }
    if (threadIdx.x == kScanT - 1) block_tot[blockIdx.x] = incl;
}

// Single block: exclusive offsets of the block totals (sequential per thread chunk).
__global__ void k_scan_totals(double* tot, int nb)
{
    __shared__ double sh[kScanT];
    int per = (nb + kScanT - 1) / kScanT;
    int b0 = threadIdx.x * per;
    double run = 0.0;
    for (int b = b0; b < b0 + per && b < nb; ++b) run += tot[b];
    double incl = block_inclusive_scan(run, sh);
    double off = incl - run;
    for (int b = b0; b < b0 + per && b < nb; ++b) {
        double t = tot[b];
        tot[b] = off;
        off += t;
    }
}

__global__ void k_scan_total(const double* out, int n, double* offs, int nb, int* bad)
{
    double total = out[n - 1] + offs[(n - 1) / kScanChunk];
    offs[nb] = total;
    if (!(total > 0.0)) atomicOr(bad, 2);
}

__global__ void k_scan_finish(double* out, int n, const double* offs, int nb)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n) return;
    double total = offs[nb];
    if (!(total > 0.0)) return;
    out[i] = (out[i] + offs[i / kScanChunk]) / total;
}

__global__ void k_add_counters(unsigned long long* out, const unsigned long long* in, int n)
{
    int i = threadIdx.x;
    if (i < n && in[i]) atomicAdd(out + i, in[i]);   // runs on other streams may add too
}

__global__ void k_add_counters_batch(unsigned long long* const* dst, const unsigned long long* src, int n_models)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_models * ST_N) return;
    const unsigned long long v = src[i];
    if (v) atomicAdd(dst[i / ST_N] + (i % ST_N), v);
}

}  // namespace

cudaError_t add_counters_batch(unsigned long long* const* dst, const unsigned long long* src, int n_models,
                               cudaStream_t s)
{
    const int n = n_models * ST_N;
    k_add_counters_batch<<<(n + 127) / 128, 128, 0, s>>>(dst, src, n_models);
    return cudaGetLastError();
}

size_t line_tables_work_doubles() { return 64 + (size_t)kRnX * (kUsNu - 1); }

cudaError_t build_line_tables(double a, const LineTables& T, bool with_r, cudaStream_t s)
{
    const int N = kWeidemanN;
    const double L = weideman_L(N);
    double* coef = T.work;
    k_weideman<<<1, 64, 0, s>>>(coef, N, L);
    k_voigt<<<(kVoigtN + 255) / 256, 256, 0, s>>>(a, coef, N, L, T.voigt_lnH, T.H0);
    k_usampler<<<kUsNx, 256, 0, s>>>(a, T.us_x, T.us_lncdf, T.us_guide);
    if (with_r) {
        double* p = T.work + 64;
        k_rmasses<<<(kRnX + 127) / 128, 128, 0, s>>>(a, p);
        k_rtable<<<(unsigned)((kRtabElems + 255) / 256), 256, 0, s>>>(p, T.rtab);
        if (T.rquad) k_rquad<<<(unsigned)((kRquadElems + 255) / 256), 256, 0, s>>>(T.rtab, T.rquad);
    }
    return cudaGetLastError();
}

cudaError_t build_voigt2d(float* out, double* work, cudaStream_t s)
{
    const int N = kWeidemanN;
    const double L = weideman_L(N);
    k_weideman<<<1, 64, 0, s>>>(work, N, L);
    k_voigt2d<<<(kV2Na * kV2Nx + 255) / 256, 256, 0, s>>>(work, N, L, out);
    return cudaGetLastError();
}

cudaError_t derive_fields(const FieldArgs& F, cudaStream_t s)
{
    k_fields<<<(F.ncell + 255) / 256, 256, 0, s>>>(F);
    return cudaGetLastError();
}

cudaError_t validate_field(const float* f, int n, bool allow_negative, int* bad, cudaStream_t s)
{
    if (!f || n <= 0) return cudaSuccess;
    k_validate<<<(n + 255) / 256, 256, 0, s>>>(f, n, allow_negative ? 1 : 0, bad);
    return cudaGetLastError();
}

size_t emission_cdf_work_doubles(int n) { return (size_t)(n + kScanChunk - 1) / kScanChunk + 1; }

cudaError_t emission_cdf(const float* rate, int n, double* cdf, double* work, size_t work_doubles,
                         int* bad, cudaStream_t s)
{
    int nb = (n + kScanChunk - 1) / kScanChunk;
    if ((size_t)nb + 1 > work_doubles) return cudaErrorInvalidValue;
    k_scan_local<<<nb, kScanT, 0, s>>>(rate, n, cdf, work, bad);
    k_scan_totals<<<1, kScanT, 0, s>>>(work, nb);
    k_scan_total<<<1, 1, 0, s>>>(cdf, n, work, nb, bad);
    k_scan_finish<<<(n + 255) / 256, 256, 0, s>>>(cdf, n, work, nb);
    return cudaGetLastError();
}

cudaError_t add_counters(unsigned long long* out, const unsigned long long* in, int n, cudaStream_t s)
{
    k_add_counters<<<1, 32, 0, s>>>(out, in, n);
    return cudaGetLastError();
}

}  // namespace krl
