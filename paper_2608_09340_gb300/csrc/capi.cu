// C ABI of libkrl (declared in include/krl.h): grid and line objects, the
// packet-run entry point and tally readout. Host code only; every step of
// the walk runs in the kernels of transport.cu and tables.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "krl_internal.cuh"

using namespace krl;

struct krl_grid {
    int nx = 0, ny = 0, nz = 0, ncell = 0;
    double cell_cm = 0.0;
    unsigned periodic = 0;
    int opacity_kind = 0;
    double T_K = 0.0;
    int device = 0;
    int num_sms = 0;
    // owned copies of the fields
    float* opacity = nullptr;
    float* vel[3] = {nullptr, nullptr, nullptr};
    float* n_coll = nullptr;
    float* tau_abs = nullptr;            // continuum absorption per cell width, or NULL
    bool has_vel = false;
    // line
    bool line_ok = false;
    unsigned line_gen = 0;     // bumped by every krl_line_set (batches check it)
    krl_line_desc line{};
    krl_line_info info{};
    bool has_rtab = false;
    float4* cells = nullptr;
    float* eps = nullptr;
    float* src_rate = nullptr;
    double* src_cdf = nullptr;
    LineTables tab{};
    // tallies
    double* spec_w = nullptr;
    unsigned long long* spec_c = nullptr;
    unsigned long long* scat = nullptr;
    double* exc = nullptr;
    double* J = nullptr;
    float* emiss = nullptr;
    double* absw = nullptr;                   // [ncell] weight absorbed by the continuum
    unsigned long long* stats = nullptr;      // cumulative [ST_N]
    // scratch: a ring of per-run slots so that runs on different streams can
    // be in flight together (each slot: work counter + ST_N run counters)
    unsigned long long* run_stats = nullptr;  // [kSlots][ST_N]
    unsigned long long* next = nullptr;       // [kSlots] work counters
    std::atomic<unsigned> run_seq{0};         // runs take slots round robin
    // A slot is reused by every 8th run: the next user waits (on its own
    // stream) for the event recorded after the previous user's last read of
    // the slot; the slot's mutex orders that wait and record on the host.
    cudaEvent_t slot_ev[8] = {};
    std::mutex slot_mu[8];
    int* bad = nullptr;                       // validation flags
    double* scan_work = nullptr;
    size_t scan_work_n = 0;
    // level iteration scratch
    double* lv_gamma = nullptr;          // [kMaxTrans][ncell]
    double* lv_pops0 = nullptr;          // [ncell][kMaxLevels] frozen emission populations
    float* lv_rate = nullptr;            // [ncell] source rate of the current line
    double* lv_total = nullptr;          // [0]: emission total; then its partial sums
    unsigned long long* lv_change = nullptr;
    // line-profile modes 1 and 3 (krl_line_desc.ph_mode)
    float* voigt2d = nullptr;            // [kV2Na][kV2Nx], built once on first use
    int v2_row = 0;
    double v2_w = 0.0;
    double u0 = 0.0;
};

namespace {

thread_local char g_err[512] = "";

krl_status fail(krl_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

krl_status cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) return fail(KRL_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(KRL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define KRL_CUDA(call, what)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n)
{
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    return cudaMalloc((void**)p, n * sizeof(T));
}

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void free_line(krl_grid* g)
{
    dfree(g->cells);
    dfree(g->eps);
    dfree(g->src_rate);
    dfree(g->src_cdf);
    dfree(g->tab.voigt_lnH);
    dfree(g->tab.H0);
    dfree(g->tab.us_x);
    dfree(g->tab.us_lncdf);
    dfree(g->tab.us_guide);
    dfree(g->tab.rtab);
    dfree(g->tab.rquad);
    dfree(g->tab.work);
    dfree(g->spec_w);
    dfree(g->spec_c);
    dfree(g->scat);
    dfree(g->exc);
    dfree(g->J);
    dfree(g->emiss);
    dfree(g->scan_work);
    g->line_ok = false;
}

constexpr int kSlots = 8;   // runs that may be in flight at once on one grid

// Physical constants (CGS, CODATA 2018).
constexpr double kKB = 1.380649e-16;
constexpr double kC = 2.99792458e10;
constexpr double kAmu = 1.66053906660e-24;
constexpr double kPiD = 3.14159265358979323846;

size_t tally_elems(const krl_grid* g, krl_tally_kind k, size_t* esz)
{
    const krl_line_desc& L = g->line;
    size_t nb = (size_t)L.spec_nbins + 2;
    switch (k) {
    case KRL_OUT_SPEC_W: *esz = 8; return g->spec_w ? nb : 0;
    case KRL_OUT_SPEC_N: *esz = 8; return g->spec_c ? nb : 0;
    case KRL_OUT_SCATMAP: *esz = 8; return g->scat ? (size_t)g->ncell : 0;
    case KRL_OUT_EXC: *esz = 8; return g->exc ? (size_t)g->ncell : 0;
    case KRL_OUT_J: *esz = 8; return g->J ? (size_t)g->ncell * L.n_ch : 0;
    case KRL_OUT_EMISS: *esz = 4; return g->emiss ? (size_t)L.n_cam * g->ncell * L.n_ch : 0;
    case KRL_OUT_STATS: *esz = 8; return g->stats ? (size_t)ST_N : 0;
    case KRL_OUT_ABSW: *esz = 8; return g->absw ? (size_t)g->ncell : 0;
    case KRL_OUT_VOIGT: *esz = 4; return g->tab.voigt_lnH ? (size_t)kVoigtN : 0;
    case KRL_OUT_US_X: *esz = 4; return g->tab.us_x ? (size_t)kUsNx : 0;
    case KRL_OUT_US_LNCDF: *esz = 4; return g->tab.us_lncdf ? (size_t)kUsNx * kUsNu : 0;
    case KRL_OUT_RTAB: *esz = 4; return g->tab.rtab ? kRtabElems : 0;
    case KRL_OUT_CELLS: *esz = 16; return g->cells ? (size_t)g->ncell : 0;
    case KRL_OUT_EPS: *esz = 4; return g->eps ? (size_t)g->ncell : 0;
    case KRL_OUT_SRC_CDF: *esz = 8; return g->src_cdf ? (size_t)g->ncell : 0;
    case KRL_OUT_H0: *esz = 4; return g->tab.H0 ? 1 : 0;
    case KRL_OUT_VOIGT2D: *esz = 4; return g->voigt2d ? (size_t)kV2Na * kV2Nx : 0;
    }
    *esz = 0;
    return 0;
}

const void* tally_ptr(const krl_grid* g, krl_tally_kind k)
{
    switch (k) {
    case KRL_OUT_SPEC_W: return g->spec_w;
    case KRL_OUT_SPEC_N: return g->spec_c;
    case KRL_OUT_SCATMAP: return g->scat;
    case KRL_OUT_EXC: return g->exc;
    case KRL_OUT_J: return g->J;
    case KRL_OUT_EMISS: return g->emiss;
    case KRL_OUT_STATS: return g->stats;
    case KRL_OUT_ABSW: return g->absw;
    case KRL_OUT_VOIGT: return g->tab.voigt_lnH;
    case KRL_OUT_US_X: return g->tab.us_x;
    case KRL_OUT_US_LNCDF: return g->tab.us_lncdf;
    case KRL_OUT_RTAB: return g->tab.rtab;
    case KRL_OUT_CELLS: return g->cells;
    case KRL_OUT_EPS: return g->eps;
    case KRL_OUT_SRC_CDF: return g->src_cdf;
    case KRL_OUT_H0: return g->tab.H0;
    case KRL_OUT_VOIGT2D: return g->voigt2d;
    }
    return nullptr;
}

krl_status zero_tallies(krl_grid* g, cudaStream_t s)
{
    for (int k = 0; k <= (int)KRL_OUT_ABSW; ++k) {
        size_t esz;
        size_t n = tally_elems(g, (krl_tally_kind)k, &esz);
        if (n) KRL_CUDA(cudaMemsetAsync((void*)tally_ptr(g, (krl_tally_kind)k), 0, n * esz, s), "zero tallies");
    }
    return KRL_OK;
}


unsigned features_of(const krl_grid* g)
{
    const krl_line_desc& L = g->line;
    unsigned f = 0;
    if (g->has_vel) f |= F_VEL;
    if (L.tally_flags & KRL_TALLY_SCATMAP) f |= F_SCAT;
    if ((L.tally_flags & (KRL_TALLY_EXC | KRL_TALLY_J | KRL_TALLY_EMISS)) || g->eps || g->tau_abs) f |= F_RICH;
    return f;
}

// The walk's argument block for one grid (work counter and run counters are
// filled in by the caller).
void fill_args(const krl_grid* g, TransportArgs& A, uint64_t n, uint64_t first_id, uint64_t seed, const krl_tune& T,
               krl_packet_record* records)
{
    const krl_line_desc& L = g->line;
    unsigned rich = L.tally_flags & (KRL_TALLY_EXC | KRL_TALLY_J | KRL_TALLY_EMISS);
    if (g->eps) rich |= kRichEps;
    A.cells = g->cells;
    A.eps = g->eps;
    A.nx = g->nx;
    A.ny = g->ny;
    A.nz = g->nz;
    A.ncell = g->ncell;
    A.periodic = g->periodic;
    A.a = g->info.a;
    A.H0 = g->tab.H0;
    A.voigt_lnH = g->tab.voigt_lnH;
    A.us_x = g->tab.us_x;
    A.us_lncdf = g->tab.us_lncdf;
    A.us_guide = g->tab.us_guide;
    A.rtab = g->tab.rtab;
    A.rquad = g->tab.rquad;
    A.src_kind = L.src_kind;
    A.src_profile = L.src_profile;
    A.src_axis = L.src_axis;
    A.band_axis = L.band_axis;
    for (int k = 0; k < 3; ++k) A.src_pos[k] = L.src_pos[k];
    A.src_plane = L.src_plane;
    A.band_lo = L.band_lo;
    A.band_hi = L.band_hi;
    A.src_cdf = g->src_cdf;
    A.spec_lo = L.spec_xmin;
    A.spec_hi = L.spec_xmax;
    A.spec_n = L.spec_nbins;
    A.n_ch = L.n_ch;
    A.ch_x0 = L.ch_vmin_cms / g->info.b_cms;
    A.ch_dx = L.ch_dv_cms / g->info.b_cms;
    A.n_cam = L.n_cam;
    for (int m = 0; m < L.n_cam; ++m) {
        double th = L.cam_theta[m], ph = L.cam_phi[m];
        A.cam[m][0] = (float)(sin(th) * cos(ph));
        A.cam[m][1] = (float)(sin(th) * sin(ph));
        A.cam[m][2] = (float)cos(th);
    }
    A.rich = rich;
    A.spec_w = g->spec_w;
    A.spec_c = g->spec_c;
    A.scat = g->scat;
    A.exc = g->exc;
    A.J = g->J;
    A.emiss = g->emiss;
    A.rec = records;
    A.first = first_id;
    A.n = n;
    A.k0 = (unsigned)(seed & 0xffffffffu);
    A.k1 = (unsigned)(seed >> 32);
    A.keys = round_keys(seed);
    A.max_iters = T.max_iters;
    A.max_iters32 = (unsigned)T.max_iters;        // resolve_tune keeps it below 2^32
    A.refill_min = T.refill_min;
    A.tau_abs = g->tau_abs;
    A.absw = g->absw;
    A.ph_mode = g->line.ph_mode;
    A.voigt2d = g->voigt2d;
    A.v2_row = g->v2_row;
    A.v2_w = g->v2_w;
    A.u0 = g->u0;
}

// Crossing point u0 of the ph_mode 3 blend: the outer root of
// g(u) = -u^2 - ln(a / (sqrt(pi) (u^2 + a^2))) (core = wing), bracketed by
// [sqrt(1 - a^2), 30], where g has its maximum and is negative; found by
// bisection to the last bit. False when core and wing do not cross.
bool blend_crossing(double a, double* u0)
{
    if (!(a > 0.0 && a < 1.0)) return false;
    auto gf = [a](double u) { return -u * u - log(a / (sqrt(kPiD) * (u * u + a * a))); };
    double lo = sqrt(1.0 - a * a), hi = 30.0;
    if (!(gf(lo) > 0.0)) return false;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (gf(mid) > 0.0) lo = mid;
        else hi = mid;
    }
    *u0 = 0.5 * (lo + hi);
    return true;
}

krl_status resolve_tune(const krl_tune* tune, krl_tune& T)
{
    T = krl_tune{KRL_PREC_FP32, 0, 0, 1, 0xFFFFFFFFull, 0, KRL_TABLES_SHARED};
    if (tune) {
        if (tune->table_space != KRL_TABLES_SHARED && tune->table_space != KRL_TABLES_CONSTANT)
            return fail(KRL_ERR_ARG, "unknown table_space %d", tune->table_space);
        T.table_space = tune->table_space;
        if (tune->emiss_records < -1 || tune->emiss_records > (1ll << 36))
            return fail(KRL_ERR_ARG, "emiss_records must be in [-1, 2^36]");
        T.emiss_records = tune->emiss_records;
        if (tune->precision != KRL_PREC_FP32 && tune->precision != KRL_PREC_FP64)
            return fail(KRL_ERR_ARG, "unknown precision");
        T.precision = tune->precision;
        if (tune->block) T.block = tune->block;
        if (tune->ctas_per_sm) T.ctas_per_sm = tune->ctas_per_sm;
        if (tune->refill_min) T.refill_min = tune->refill_min;
        if (tune->max_iters > 0xFFFFFFFFull)
            return fail(KRL_ERR_ARG, "max_iters must be at most 2^32 - 1 (the walk counts events in 32 bits)");
        if (tune->max_iters) T.max_iters = tune->max_iters;
    }
    if (T.block && (T.block < 32 || T.block > 512 || T.block % 32))
        return fail(KRL_ERR_ARG, "block must be a multiple of 32 in [32, 512]");
    if (T.refill_min < 1 || T.refill_min > 32) return fail(KRL_ERR_ARG, "refill_min must be in [1, 32]");
    return KRL_OK;
}

}  // namespace

namespace krl {
// Lets other translation units report through krl_last_error().
void set_last_error(const char* msg)
{
    snprintf(g_err, sizeof(g_err), "%s", msg);
}
}  // namespace krl

extern "C" {

const char* krl_last_error(void) { return g_err; }

int krl_version(void) { return 500; }       // 0.5.0: records carry scat_cells; krl_tune.table_space

krl_status krl_grid_create(krl_grid** out, const krl_grid_desc* d, krl_stream st)
{
    cudaStream_t s = (cudaStream_t)st;
    if (!out || !d) return fail(KRL_ERR_ARG, "krl_grid_create: NULL argument");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(KRL_ERR_ARG, "grid dimensions must be >= 1");
    long long nc = (long long)d->nx * d->ny * d->nz;
    if (nc >= (1ll << 31)) return fail(KRL_ERR_ARG, "grid has too many cells (%lld)", nc);
    if (!(d->cell_cm > 0.0) || !isfinite(d->cell_cm)) return fail(KRL_ERR_ARG, "cell_cm must be > 0");
    if (!(d->T_K > 0.0) || !isfinite(d->T_K)) return fail(KRL_ERR_ARG, "T_K must be > 0");
    if (d->opacity_kind != KRL_OPACITY_TAU && d->opacity_kind != KRL_OPACITY_NL)
        return fail(KRL_ERR_ARG, "unknown opacity_kind %d", d->opacity_kind);
    if (!d->opacity) return fail(KRL_ERR_ARG, "opacity field is required");
    if (d->boundary_flags & ~7u) return fail(KRL_ERR_ARG, "unknown boundary flag bits");
    krl_grid* g = new (std::nothrow) krl_grid();
    if (!g) return fail(KRL_ERR_OOM, "host allocation failed");
    g->nx = d->nx;
    g->ny = d->ny;
    g->nz = d->nz;
    g->ncell = (int)nc;
    g->cell_cm = d->cell_cm;
    g->periodic = d->boundary_flags;
    g->opacity_kind = d->opacity_kind;
    g->T_K = d->T_K;
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    size_t n = (size_t)nc;
    cudaError_t e = dalloc(&g->opacity, n);
    const float* src[3] = {d->vx, d->vy, d->vz};
    g->has_vel = d->vx || d->vy || d->vz;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (src[k]) e = dalloc(&g->vel[k], n);
    if (e == cudaSuccess && d->n_coll) e = dalloc(&g->n_coll, n);
    if (e == cudaSuccess && d->tau_abs) e = dalloc(&g->tau_abs, n);
    if (e == cudaSuccess && d->tau_abs) e = dalloc(&g->absw, n);
    if (e == cudaSuccess) e = dalloc(&g->stats, ST_N);
    if (e == cudaSuccess) e = dalloc(&g->run_stats, (size_t)kSlots * ST_N);
    if (e == cudaSuccess) e = dalloc(&g->next, (size_t)kSlots);
    if (e == cudaSuccess) e = dalloc(&g->bad, 1);
    for (int k = 0; k < kSlots && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&g->slot_ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->opacity, d->opacity, n * 4, cudaMemcpyDeviceToDevice, s);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (src[k]) e = cudaMemcpyAsync(g->vel[k], src[k], n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d->n_coll) e = cudaMemcpyAsync(g->n_coll, d->n_coll, n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d->tau_abs)
        e = cudaMemcpyAsync(g->tau_abs, d->tau_abs, n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && g->absw) e = cudaMemsetAsync(g->absw, 0, n * 8, s);
    if (e == cudaSuccess) e = validate_field(g->opacity, g->ncell, false, g->bad, s);
    if (e == cudaSuccess && g->tau_abs) e = validate_field(g->tau_abs, g->ncell, false, g->bad, s);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (g->vel[k]) e = validate_field(g->vel[k], g->ncell, true, g->bad, s);
    if (e == cudaSuccess && g->n_coll) e = validate_field(g->n_coll, g->ncell, false, g->bad, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->stats, 0, ST_N * 8, s);
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, g->bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        krl_grid_destroy(g);
        return cuda_fail(e, "krl_grid_create");
    }
    if (bad) {
        krl_grid_destroy(g);
        return fail(KRL_ERR_NUMERIC, "grid field holds NaN/Inf or a negative opacity/density/absorption");
    }
    *out = g;
    return KRL_OK;
}

krl_status krl_grid_destroy(krl_grid* g)
{
    if (!g) return KRL_OK;
    cudaDeviceSynchronize();
    free_line(g);
    dfree(g->opacity);
    for (int k = 0; k < 3; ++k) dfree(g->vel[k]);
    dfree(g->n_coll);
    dfree(g->tau_abs);
    dfree(g->absw);
    dfree(g->lv_gamma);
    dfree(g->lv_pops0);
    dfree(g->lv_rate);
    dfree(g->lv_total);
    dfree(g->lv_change);
    dfree(g->voigt2d);
    dfree(g->stats);
    dfree(g->run_stats);
    dfree(g->next);
    dfree(g->bad);
    for (int k = 0; k < kSlots; ++k)
        if (g->slot_ev[k]) cudaEventDestroy(g->slot_ev[k]);
    delete g;
    return KRL_OK;
}

krl_status krl_line_set(krl_grid* g, const krl_line_desc* d, krl_stream st)
{
    cudaStream_t s = (cudaStream_t)st;
    if (!g || !d) return fail(KRL_ERR_ARG, "krl_line_set: NULL argument");
    if (!(d->nu0_hz > 0) || !(d->mass_amu > 0) || !(d->A_ul > 0) || !(d->g_u > 0) || !(d->g_l > 0))
        return fail(KRL_ERR_ARG, "line constants must be > 0");
    if (d->k_ul < 0 || !isfinite(d->k_ul)) return fail(KRL_ERR_ARG, "k_ul must be >= 0");
    if (d->src_kind < KRL_SRC_POINT || d->src_kind > KRL_SRC_VOLUME) return fail(KRL_ERR_ARG, "unknown src_kind");
    if (d->src_profile != KRL_PROFILE_LINE_CENTRE && d->src_profile != KRL_PROFILE_GAUSSIAN)
        return fail(KRL_ERR_ARG, "unknown src_profile");
    if ((d->src_kind == KRL_SRC_PLANE || d->src_kind == KRL_SRC_BEAM) && (d->src_axis < 0 || d->src_axis > 2))
        return fail(KRL_ERR_ARG, "src_axis must be 0, 1 or 2");
    if (d->src_kind == KRL_SRC_BEAM && d->band_axis >= 0 &&
        (d->band_axis > 2 || d->band_axis == d->src_axis || !(d->band_hi >= d->band_lo)))
        return fail(KRL_ERR_ARG, "bad beam band");
    if (d->src_kind == KRL_SRC_VOLUME && !d->src_rate) return fail(KRL_ERR_ARG, "volume source needs src_rate");
    for (int k = 0; k < 3; ++k)
        if (!isfinite(d->src_pos[k])) return fail(KRL_ERR_ARG, "src_pos must be finite");
    if (d->spec_nbins < 1 || !(d->spec_xmax > d->spec_xmin)) return fail(KRL_ERR_ARG, "bad spectrum binning");
    if (d->tally_flags & ~15u) return fail(KRL_ERR_ARG, "unknown tally flag bits");
    if (d->ph_mode < 0 || d->ph_mode > 3) return fail(KRL_ERR_ARG, "ph_mode must be 0..3");
    bool need_ch = d->tally_flags & (KRL_TALLY_J | KRL_TALLY_EMISS);
    if (need_ch && (d->n_ch < 1 || !(d->ch_dv_cms > 0))) return fail(KRL_ERR_ARG, "channels need n_ch >= 1, dv > 0");
    if ((d->tally_flags & KRL_TALLY_EMISS) && (d->n_cam < 1 || d->n_cam > KRL_MAX_CAMERAS))
        return fail(KRL_ERR_ARG, "emissivity needs 1..%d cameras", KRL_MAX_CAMERAS);

    free_line(g);
    KRL_CUDA(cudaMemsetAsync(g->bad, 0, sizeof(int), s), "krl_line_set");
    krl_line_desc L = *d;
    // keep a channel grid for the ray trace even without J / emissivity tallies
    if (!need_ch && !(d->n_ch >= 1 && d->ch_dv_cms > 0)) L.n_ch = 0;
    if (!(L.tally_flags & KRL_TALLY_EMISS)) L.n_cam = 0;
    if (L.ph_mode == 0) L.ph_mode = 2;
    g->line = L;

    // scalar line constants (Sec. 2.1, Eq. xdef, Eq. sigma0)
    krl_line_info I{};
    I.b_cms = sqrt(2.0 * kKB * g->T_K / (L.mass_amu * kAmu));
    I.nu_D_hz = L.nu0_hz * I.b_cms / kC;
    I.a = L.a_fixed > 0 ? L.a_fixed : L.A_ul / (4.0 * kPiD * I.nu_D_hz);
    I.sigma0_cm2 = (L.g_u / L.g_l) * L.A_ul * kC * kC * kC / (8.0 * pow(kPiD, 1.5) * pow(L.nu0_hz, 3) * I.b_cms);
    I.ncell = g->ncell;
    g->info = I;
    if (L.ph_mode == 1) {
        if (!(I.a >= pow(10.0, kV2LaMin) && I.a <= pow(10.0, kV2LaMax))) {
            free_line(g);
            return fail(KRL_ERR_ARG, "ph_mode 1 needs 1e-6 <= a <= 1 (a = %g)", I.a);
        }
        const double s2 = (log10(I.a) - kV2LaMin) * ((kV2Na - 1) / (kV2LaMax - kV2LaMin));
        int j = (int)floor(s2);
        j = j < 0 ? 0 : (j > kV2Na - 2 ? kV2Na - 2 : j);
        g->v2_row = j;
        g->v2_w = s2 - j;
    } else if (L.ph_mode == 3) {
        if (!blend_crossing(I.a, &g->u0)) {
            free_line(g);
            return fail(KRL_ERR_ARG, "ph_mode 3: core and wing do not cross at a = %g", I.a);
        }
    }

    const size_t n = (size_t)g->ncell;
    const bool with_r = (L.tally_flags & KRL_TALLY_EMISS) != 0;
    const bool with_eps = L.k_ul > 0 && g->n_coll;
    cudaError_t e = dalloc(&g->cells, n);
    if (e == cudaSuccess && with_eps) e = dalloc(&g->eps, n);
    if (e == cudaSuccess) e = dalloc(&g->tab.voigt_lnH, (size_t)kVoigtN);
    if (e == cudaSuccess) e = dalloc(&g->tab.H0, 1);
    if (e == cudaSuccess) e = dalloc(&g->tab.us_x, (size_t)kUsNx);
    if (e == cudaSuccess) e = dalloc(&g->tab.us_lncdf, (size_t)kUsNx * kUsNu);
    if (e == cudaSuccess) e = dalloc(&g->tab.us_guide, (size_t)kUsNx * kGuideN);
    if (e == cudaSuccess && with_r) e = dalloc(&g->tab.rtab, kRtabElems);
    if (e == cudaSuccess && with_r) e = dalloc(&g->tab.rquad, kRquadElems);
    if (e == cudaSuccess) e = dalloc(&g->tab.work, line_tables_work_doubles());
    if (e == cudaSuccess) e = dalloc(&g->spec_w, (size_t)L.spec_nbins + 2);
    if (e == cudaSuccess) e = dalloc(&g->spec_c, (size_t)L.spec_nbins + 2);
    if (e == cudaSuccess && (L.tally_flags & KRL_TALLY_SCATMAP)) e = dalloc(&g->scat, n);
    if (e == cudaSuccess && (L.tally_flags & KRL_TALLY_EXC)) e = dalloc(&g->exc, n);
    if (e == cudaSuccess && (L.tally_flags & KRL_TALLY_J)) e = dalloc(&g->J, n * L.n_ch);
    if (e == cudaSuccess && with_r) e = dalloc(&g->emiss, (size_t)L.n_cam * n * L.n_ch);
    if (e == cudaSuccess && L.src_kind == KRL_SRC_VOLUME) {
        e = dalloc(&g->src_rate, n);
        if (e == cudaSuccess) e = dalloc(&g->src_cdf, n);
        g->scan_work_n = emission_cdf_work_doubles(g->ncell);
        if (e == cudaSuccess) e = dalloc(&g->scan_work, g->scan_work_n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->src_rate, L.src_rate, n * 4, cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) {
        free_line(g);
        return cuda_fail(e, "krl_line_set allocation");
    }
    g->has_rtab = with_r;
    g->line.src_rate = g->src_rate;

    FieldArgs F{};
    F.ncell = g->ncell;
    F.opacity_kind = g->opacity_kind;
    F.opacity = g->opacity;
    F.vx = g->vel[0];
    F.vy = g->vel[1];
    F.vz = g->vel[2];
    F.n_coll = g->n_coll;
    F.tau_scale = g->opacity_kind == KRL_OPACITY_NL ? I.sigma0_cm2 * g->cell_cm : 1.0;
    F.inv_b = 1.0 / I.b_cms;
    F.k_ul = L.k_ul;
    F.A_ul = L.A_ul;
    F.cells = g->cells;
    F.eps = g->eps;
    e = derive_fields(F, s);
    if (e == cudaSuccess) e = build_line_tables(I.a, g->tab, with_r, s);
    if (e == cudaSuccess && L.ph_mode == 1 && !g->voigt2d) {
        e = dalloc(&g->voigt2d, (size_t)kV2Na * kV2Nx);
        if (e == cudaSuccess) e = build_voigt2d(g->voigt2d, g->tab.work, s);
    }
    if (e == cudaSuccess && L.src_kind == KRL_SRC_VOLUME)
        e = emission_cdf(g->src_rate, g->ncell, g->src_cdf, g->scan_work, g->scan_work_n, g->bad, s);
    if (e != cudaSuccess) {
        free_line(g);
        return cuda_fail(e, "krl_line_set kernels");
    }
    krl_status zs = zero_tallies(g, s);
    if (zs != KRL_OK) return zs;
    // H(a, 0) for krl_line_info_get (small synchronous copy on this stream)
    float h0 = 0.0f;
    e = cudaMemcpyAsync(&h0, g->tab.H0, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "krl_line_set");
    int bad = 0;
    cudaMemcpy(&bad, g->bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (bad & 2) {
        free_line(g);
        return fail(KRL_ERR_ARG, "volume source rate sums to zero");
    }
    if (bad) {
        free_line(g);
        return fail(KRL_ERR_NUMERIC, "volume source rate holds NaN/Inf or a negative value");
    }
    g->info.H0 = h0;
    g->line_ok = true;
    ++g->line_gen;
    return KRL_OK;
}

krl_status krl_line_info_get(const krl_grid* g, krl_line_info* out)
{
    if (!g || !out) return fail(KRL_ERR_ARG, "krl_line_info_get: NULL argument");
    if (!g->line_ok) return fail(KRL_ERR_STATE, "no line set");
    *out = g->info;
    return KRL_OK;
}

krl_status krl_run_packets(krl_grid* g, uint64_t n, uint64_t first_id, uint64_t seed, const krl_tune* tune,
                           krl_packet_record* records, krl_run_stats* stats, krl_stream st)
{
    cudaStream_t s = (cudaStream_t)st;
    if (!g) return fail(KRL_ERR_ARG, "krl_run_packets: NULL grid");
    if (!g->line_ok) return fail(KRL_ERR_STATE, "krl_run_packets before krl_line_set");
    krl_tune T;
    krl_status ts = resolve_tune(tune, T);
    if (ts != KRL_OK) return ts;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (n == 0) return KRL_OK;

    const unsigned f = features_of(g);
    const int maxb = transport_max_block(T.precision, f);
    if (!tune || !tune->block) T.block = maxb;
    else if (T.block > maxb) return fail(KRL_ERR_ARG, "block %d exceeds %d for this walk", T.block, maxb);
    // constant-bank tables: profile mode 2, FP32 walk (internal mode 4)
    int mode = g->line.ph_mode;
    if (T.table_space == KRL_TABLES_CONSTANT) {
        if (mode != 2 || T.precision != KRL_PREC_FP32)
            return fail(KRL_ERR_ARG, "table_space = constant needs ph_mode 2 and the FP32 walk");
        mode = 4;
    }
    int occ = transport_occupancy(T.precision, f, T.block, mode);
    if (occ < 1) return fail(KRL_ERR_CUDA, "transport kernel cannot be resident at block %d", T.block);
    int per_sm = T.ctas_per_sm > 0 ? (T.ctas_per_sm < occ ? T.ctas_per_sm : occ) : occ;
    int grid = g->num_sms * per_sm;

    TransportArgs A{};
    fill_args(g, A, n, first_id, seed, T, records);
    A.ph_mode = mode;
    const int slot = (int)(g->run_seq.fetch_add(1u, std::memory_order_relaxed) % kSlots);
    unsigned long long* slot_stats = g->run_stats + (size_t)slot * ST_N;
    unsigned long long* slot_next = g->next + slot;
    A.stats = slot_stats;
    A.next = slot_next;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    KRL_CUDA(cudaStreamIsCapturing(s, &cap), "krl_run_packets");
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> slot_lock(g->slot_mu[slot]);
    // the slot's previous user must have read its counters before they are
    // reset here (eager calls; a captured run keeps its slot in the graph)
    if (!capturing) KRL_CUDA(cudaStreamWaitEvent(s, g->slot_ev[slot], 0), "wait for the slot's previous run");

    KRL_CUDA(cudaMemsetAsync(slot_next, 0, sizeof(unsigned long long), s), "reset work counter");
    KRL_CUDA(cudaMemsetAsync(slot_stats, 0, ST_N * sizeof(unsigned long long), s), "reset run counters");
    // Two-stage emissivity deposit (FP32 walk): a stream-ordered segment
    // buffer for this run; without one the walk deposits every segment.
    void* segbuf = nullptr;
    if (T.precision == KRL_PREC_FP32 && g->emiss && T.emiss_records >= 0) {
        const unsigned long long lo = 1ull << 16, hi = 1ull << 25;
        unsigned long long cap = (unsigned long long)T.emiss_records;
        if (cap == 0) cap = n > hi / 64 ? hi : (n * 64 < lo ? lo : n * 64);
        if (cudaMallocAsync(&segbuf, 16 + (size_t)cap * 32, s) == cudaSuccess) {
            A.seg_count = static_cast<unsigned long long*>(segbuf);
            A.seg = reinterpret_cast<float4*>(static_cast<char*>(segbuf) + 16);
            A.seg_cap = cap;
        } else {
            (void)cudaGetLastError();
            segbuf = nullptr;
        }
    }
    cudaError_t le = cudaSuccess;
    if (segbuf) le = cudaMemsetAsync(segbuf, 0, sizeof(unsigned long long), s);
    if (le == cudaSuccess) le = launch_transport(A, T.precision, f, grid, T.block, s);
    if (le == cudaSuccess && segbuf) le = launch_emiss_deposit(A, f, g->num_sms, s);
    if (segbuf) {
        const cudaError_t fe = cudaFreeAsync(segbuf, s);
        if (le == cudaSuccess) le = fe;
    }
    if (le != cudaSuccess) return cuda_fail(le, "transport launch");
    KRL_CUDA(add_counters(g->stats, slot_stats, ST_N, s), "accumulate counters");
    unsigned long long h[ST_N];
    if (stats) KRL_CUDA(cudaMemcpyAsync(h, slot_stats, sizeof(h), cudaMemcpyDeviceToHost, s), "read counters");
    if (!capturing) KRL_CUDA(cudaEventRecord(g->slot_ev[slot], s), "release the run's slot");
    if (stats) {
        KRL_CUDA(cudaStreamSynchronize(s), "krl_run_packets");
        stats->emitted = h[ST_EMITTED];
        stats->escaped = h[ST_ESCAPED];
        stats->destroyed = h[ST_DESTROYED];
        stats->stuck = h[ST_STUCK];
        stats->scatterings = h[ST_SCAT];
        stats->crossings = h[ST_CROSS];
        stats->absorbed = h[ST_ABSORBED];
        if (h[ST_STUCK]) return fail(KRL_ERR_BUDGET, "%llu packets exhausted max_iters", h[ST_STUCK]);
    }
    return KRL_OK;
}

krl_status krl_raytrace_channels(krl_grid* g, const krl_raytrace_desc* d, float* maps, krl_stream st)
{
    if (!g || !d || !maps) return fail(KRL_ERR_ARG, "krl_raytrace_channels: NULL argument");
    if (!g->line_ok) return fail(KRL_ERR_STATE, "krl_raytrace_channels before krl_line_set");
    if (g->line.ph_mode != 2) return fail(KRL_ERR_ARG, "the ray trace uses the ph_mode 2 profile slice");
    const krl_line_desc& L = g->line;
    if (L.n_ch < 1 || L.n_ch > 128) return fail(KRL_ERR_ARG, "ray trace needs 1..128 line channels (line has %d)", L.n_ch);
    if (d->npix_x < 1 || d->npix_y < 1 || !(d->fov_cells > 0) || !isfinite(d->fov_cells))
        return fail(KRL_ERR_ARG, "bad image size");
    double th, ph;
    const float* em = d->emiss;
    if (d->camera >= 0) {
        if (d->camera >= L.n_cam) return fail(KRL_ERR_ARG, "camera %d not defined (line has %d)", d->camera, L.n_cam);
        th = L.cam_theta[d->camera];
        ph = L.cam_phi[d->camera];
        if (!em) {
            if (!g->emiss) return fail(KRL_ERR_STATE, "no emissivity tally on this grid");
            em = g->emiss + (size_t)d->camera * g->ncell * L.n_ch;
        }
    } else if (d->camera == -1) {
        th = d->theta;
        ph = d->phi;
        if (!em) return fail(KRL_ERR_ARG, "camera -1 needs an emissivity buffer");
        if (!isfinite(th) || !isfinite(ph)) return fail(KRL_ERR_ARG, "bad camera angles");
    } else {
        return fail(KRL_ERR_ARG, "camera must be >= -1");
    }
    RayArgs A{};
    A.cells = g->cells;
    A.tau_abs = g->tau_abs;
    A.nx = g->nx;
    A.ny = g->ny;
    A.nz = g->nz;
    A.voigt_lnH = g->tab.voigt_lnH;
    A.H0 = g->tab.H0;
    A.a = (float)g->info.a;
    A.emiss = em;
    A.jline = d->jline;
    A.n_ch = L.n_ch;
    A.ch_x0 = L.ch_vmin_cms / g->info.b_cms;
    A.ch_dx = L.ch_dv_cms / g->info.b_cms;
    A.n[0] = sin(th) * cos(ph);
    A.n[1] = sin(th) * sin(ph);
    A.n[2] = cos(th);
    A.u[0] = cos(th) * cos(ph);
    A.u[1] = cos(th) * sin(ph);
    A.u[2] = -sin(th);
    A.v[0] = -sin(ph);
    A.v[1] = cos(ph);
    A.v[2] = 0.0;
    // face ahead along -n on each axis: (1 - p) / d for d > 0, -p / d for
    // d < 0, as one FMA; an axis the ray runs parallel to (or whose inverse
    // overflows) gets a distance of 3e38, never the nearest
    for (int k = 0; k < 3; ++k) {
        const float d = (float)(-A.n[k]);
        const float inv = 1.0f / d;
        A.dirf[k] = d;
        if (d != 0.0f && fabsf(inv) < 1e30f) {
            A.face_neg[k] = -inv;
            A.face_c[k] = d > 0.0f ? inv : 0.0f;
        } else {
            A.face_neg[k] = 0.0f;
            A.face_c[k] = 3.0e38f;
        }
    }
    A.centre[0] = 0.5 * g->nx;
    A.centre[1] = 0.5 * g->ny;
    A.centre[2] = 0.5 * g->nz;
    A.pix = d->fov_cells / d->npix_x;
    A.npix_x = d->npix_x;
    A.npix_y = d->npix_y;
    A.maps = maps;
    // Per-camera profile cube, stream-ordered scratch (so calls on different
    // streams never share it). Without the memory the trace evaluates the
    // profile per segment instead, with the same result.
    cudaStream_t s = (cudaStream_t)st;
    const size_t hbytes = ((size_t)g->ncell * (size_t)L.n_ch * sizeof(float) + 255) / 256 * 256;
    const size_t rbytes = (size_t)d->npix_x * (size_t)d->npix_y * 2 * sizeof(float4);
    A.hcube = nullptr;
    A.rayinit = nullptr;
    if (!d->no_scratch && cudaMallocAsync((void**)&A.hcube, hbytes + rbytes, s) != cudaSuccess) {
        (void)cudaGetLastError();
        A.hcube = nullptr;
    }
    if (A.hcube) A.rayinit = reinterpret_cast<float4*>(reinterpret_cast<char*>(A.hcube) + hbytes);
    cudaError_t e = launch_raytrace(A, g->num_sms, s);
    if (A.hcube) {
        cudaError_t ef = cudaFreeAsync(A.hcube, s);
        if (e == cudaSuccess) e = ef;
    }
    KRL_CUDA(e, "ray trace launch");
    return KRL_OK;
}

}  // extern "C"

struct krl_batch {
    int n = 0;
    int device = 0;
    int num_sms = 0;
    std::vector<krl_grid*> grids;
    std::vector<unsigned> gens;
    TransportArgs* h_args = nullptr;          // pinned mirror, updated by each run
    TransportArgs* d_args = nullptr;
    unsigned long long* d_counts = nullptr;   // [n] work counters, then [n][ST_N] run counters
    unsigned long long** d_dst = nullptr;     // [n] each grid's cumulative counters
    int* d_cursor = nullptr;
    unsigned features = 0;
};

extern "C" {

krl_status krl_batch_destroy(krl_batch* b)
{
    if (!b) return KRL_OK;
    cudaDeviceSynchronize();
    if (b->h_args) cudaFreeHost(b->h_args);
    dfree(b->d_args);
    dfree(b->d_counts);
    dfree(b->d_dst);
    dfree(b->d_cursor);
    delete b;
    return KRL_OK;
}

krl_status krl_batch_create(krl_batch** out, krl_grid* const* grids, int n_models, krl_stream st)
{
    if (!out || !grids || n_models < 1) return fail(KRL_ERR_ARG, "krl_batch_create: bad arguments");
    *out = nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    for (int m = 0; m < n_models; ++m) {
        if (!grids[m]) return fail(KRL_ERR_ARG, "grid %d is NULL", m);
        if (!grids[m]->line_ok) return fail(KRL_ERR_STATE, "grid %d has no line", m);
        if (grids[m]->line.ph_mode != 2) return fail(KRL_ERR_ARG, "grid %d: the batched launch runs ph_mode 2 only", m);
        if (grids[m]->device != dev) return fail(KRL_ERR_ARG, "grid %d lives on another device", m);
    }
    krl_batch* b = new (std::nothrow) krl_batch();
    if (!b) return fail(KRL_ERR_OOM, "host allocation failed");
    b->n = n_models;
    b->device = dev;
    b->num_sms = grids[0]->num_sms;
    b->grids.assign(grids, grids + n_models);
    for (int m = 0; m < n_models; ++m) {
        b->gens.push_back(grids[m]->line_gen);
        b->features |= features_of(grids[m]);
    }
    const size_t n = (size_t)n_models;
    cudaError_t e = cudaMallocHost((void**)&b->h_args, n * sizeof(TransportArgs));
    if (e == cudaSuccess) e = dalloc(&b->d_args, n);
    if (e == cudaSuccess) e = dalloc(&b->d_counts, n * (1 + ST_N));
    if (e == cudaSuccess) e = dalloc(&b->d_dst, n);
    if (e == cudaSuccess) e = dalloc(&b->d_cursor, 1);
    if (e == cudaSuccess) {
        std::vector<unsigned long long*> dst(n);
        for (size_t m = 0; m < n; ++m) dst[m] = grids[m]->stats;
        e = cudaMemcpyAsync(b->d_dst, dst.data(), n * sizeof(void*), cudaMemcpyHostToDevice, (cudaStream_t)st);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)st);
    }
    if (e != cudaSuccess) {
        krl_batch_destroy(b);
        return cuda_fail(e, "krl_batch_create");
    }
    *out = b;
    return KRL_OK;
}

krl_status krl_batch_run(krl_batch* b, const uint64_t* packets, const uint64_t* first_ids, uint64_t seed,
                         const krl_tune* tune, krl_packet_record* const* records, krl_run_stats* stats,
                         krl_stream st)
{
    cudaStream_t s = (cudaStream_t)st;
    if (!b || !packets) return fail(KRL_ERR_ARG, "krl_batch_run: NULL argument");
    for (int m = 0; m < b->n; ++m)
        if (!b->grids[m]->line_ok || b->grids[m]->line_gen != b->gens[m])
            return fail(KRL_ERR_STATE, "grid %d's line changed since krl_batch_create", m);
    krl_tune T;
    krl_status ts = resolve_tune(tune, T);
    if (ts != KRL_OK) return ts;
    if (T.table_space != KRL_TABLES_SHARED) return fail(KRL_ERR_ARG, "the batched launch stages its tables in shared memory");
    const unsigned f = b->features;
    const int maxb = transport_batch_max_block();
    if (!T.block) T.block = maxb;
    else if (T.block > maxb) return fail(KRL_ERR_ARG, "block %d exceeds %d for the batched launch", T.block, maxb);
    const int occ = transport_batch_occupancy(T.precision, f, T.block);
    if (occ < 1) return fail(KRL_ERR_CUDA, "transport kernel cannot be resident at block %d", T.block);
    const int per_sm = T.ctas_per_sm > 0 ? (T.ctas_per_sm < occ ? T.ctas_per_sm : occ) : occ;
    const int grid = b->num_sms * per_sm;
    const size_t n = (size_t)b->n;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    KRL_CUDA(cudaStreamIsCapturing(s, &cap), "krl_batch_run");
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (capturing && stats) return fail(KRL_ERR_ARG, "stats cannot be read while the stream is being captured");
    // the pinned mirror is rewritten here; wait until the previous run's copy
    // has read it (a capture records the copy instead of running it)
    if (!capturing) KRL_CUDA(cudaStreamSynchronize(s), "krl_batch_run");
    // CTAs take models in slot order: the heaviest (most packets) first, so
    // that the longest packets start early and the light models fill in
    // around them; each model keeps its own counters at its own index.
    std::vector<int> order(n);
    for (size_t m = 0; m < n; ++m) order[m] = (int)m;
    std::stable_sort(order.begin(), order.end(), [packets](int x, int y) { return packets[x] > packets[y]; });
    for (size_t k = 0; k < n; ++k) {
        const int m = order[k];
        TransportArgs& A = b->h_args[k];
        A = TransportArgs{};
        fill_args(b->grids[m], A, packets[m], first_ids ? first_ids[m] : 0, seed, T, records ? records[m] : nullptr);
        A.next = b->d_counts + m;
        A.stats = b->d_counts + n + (size_t)m * ST_N;
    }
    KRL_CUDA(cudaMemcpyAsync(b->d_args, b->h_args, n * sizeof(TransportArgs), cudaMemcpyHostToDevice, s),
             "upload model arguments");
    KRL_CUDA(cudaMemsetAsync(b->d_counts, 0, n * (1 + ST_N) * sizeof(unsigned long long), s), "reset counters");
    KRL_CUDA(cudaMemsetAsync(b->d_cursor, 0, sizeof(int), s), "reset cursor");
    BatchArgs B{b->d_args, b->n, b->d_cursor, round_keys(seed)};
    KRL_CUDA(launch_transport_batch(B, T.precision, f, grid, T.block, s), "batch launch");
    KRL_CUDA(add_counters_batch(b->d_dst, b->d_counts + n, b->n, s), "accumulate counters");
    if (stats) {
        std::vector<unsigned long long> h(n * ST_N);
        KRL_CUDA(cudaMemcpyAsync(h.data(), b->d_counts + n, h.size() * 8, cudaMemcpyDeviceToHost, s), "read counters");
        KRL_CUDA(cudaStreamSynchronize(s), "krl_batch_run");
        unsigned long long stuck = 0;
        for (size_t m = 0; m < n; ++m) {
            const unsigned long long* c = h.data() + m * ST_N;
            stats[m] = krl_run_stats{c[ST_EMITTED], c[ST_ESCAPED], c[ST_DESTROYED], c[ST_STUCK], c[ST_SCAT],
                                     c[ST_CROSS], c[ST_ABSORBED]};
            stuck += c[ST_STUCK];
        }
        if (stuck) return fail(KRL_ERR_BUDGET, "%llu packets exhausted max_iters", stuck);
    }
    return KRL_OK;
}

}  // extern "C"

namespace {

constexpr double kHPlanck = 6.62607015e-27;

krl_status level_const(const krl_grid* g, const krl_levels_desc* d, LevelConst& L)
{
    if (!d || d->n_lev < 2 || d->n_lev > kMaxLevels) return fail(KRL_ERR_ARG, "n_lev must be 2..%d", kMaxLevels);
    if (!d->n_mol) return fail(KRL_ERR_ARG, "n_mol field is required");
    L = LevelConst{};
    L.n = d->n_lev;
    L.T = g->T_K;
    for (int i = 0; i < L.n; ++i) {
        if (!(d->g[i] > 0) || !isfinite(d->E_K[i])) return fail(KRL_ERR_ARG, "bad level %d", i);
        L.E[i] = d->E_K[i];
        L.g[i] = d->g[i];
    }
    for (int l = 0; l < L.n; ++l)
        for (int u = l + 1; u < L.n; ++u) {
            if (d->A[u][l] < 0 || d->k_coll[u][l] < 0) return fail(KRL_ERR_ARG, "negative rate (%d,%d)", u, l);
            if (d->A[u][l] > 0 && !(d->E_K[u] > d->E_K[l])) return fail(KRL_ERR_ARG, "line (%d,%d) needs E_u > E_l", u, l);
            L.A[u][l] = d->A[u][l];
            L.k[u][l] = d->k_coll[u][l];
            if (d->A[u][l] > 0) {
                L.tu[L.n_trans] = u;
                L.tl[L.n_trans] = l;
                ++L.n_trans;
            }
        }
    return KRL_OK;
}

krl_status level_scratch(krl_grid* g)
{
    const size_t n = (size_t)g->ncell;
    cudaError_t e = cudaSuccess;
    if (!g->lv_gamma) e = dalloc(&g->lv_gamma, (size_t)kMaxTrans * n);
    if (e == cudaSuccess && !g->lv_pops0) e = dalloc(&g->lv_pops0, (size_t)kMaxLevels * n);
    if (e == cudaSuccess && !g->lv_rate) e = dalloc(&g->lv_rate, n);
    if (e == cudaSuccess && !g->lv_total) e = dalloc(&g->lv_total, levels_sum_scratch_doubles());
    if (e == cudaSuccess && !g->lv_change) e = dalloc(&g->lv_change, 1);
    if (e != cudaSuccess) return cuda_fail(e, "level scratch");
    return KRL_OK;
}

}  // namespace

extern "C" {

krl_status krl_levels_solve(krl_grid* g, const krl_levels_desc* d, const double* gamma, double* pops,
                            double* max_change, krl_stream st)
{
    cudaStream_t s = (cudaStream_t)st;
    if (!g || !pops) return fail(KRL_ERR_ARG, "krl_levels_solve: NULL argument");
    LevelConst L;
    krl_status ls = level_const(g, d, L);
    if (ls != KRL_OK) return ls;
    if (L.n_trans > 0 && !gamma) return fail(KRL_ERR_ARG, "gamma is required when the levels have lines");
    ls = level_scratch(g);
    if (ls != KRL_OK) return ls;
    KRL_CUDA(cudaMemsetAsync(g->lv_change, 0, sizeof(unsigned long long), s), "levels");
    KRL_CUDA(levels_solve(L, gamma, g->ncell, g->n_coll, d->n_mol, pops, g->lv_change, s), "levels solve");
    if (max_change) {
        unsigned long long bits = 0;
        KRL_CUDA(cudaMemcpyAsync(&bits, g->lv_change, 8, cudaMemcpyDeviceToHost, s), "levels");
        KRL_CUDA(cudaStreamSynchronize(s), "levels");
        memcpy(max_change, &bits, 8);
    }
    return KRL_OK;
}

krl_status krl_levels_iterate(krl_grid* g, const krl_levels_desc* d, int n_iter, uint64_t packets_per_line,
                              uint64_t seed, int init_lte, double* pops, double* max_change, krl_stream st)
{
    cudaStream_t s = (cudaStream_t)st;
    if (!g || !pops) return fail(KRL_ERR_ARG, "krl_levels_iterate: NULL argument");
    if (n_iter < 0 || packets_per_line == 0) return fail(KRL_ERR_ARG, "need n_iter >= 0 and packets_per_line > 0");
    if (g->opacity_kind != KRL_OPACITY_NL) return fail(KRL_ERR_ARG, "the grid must take its opacity as n_l");
    LevelConst L;
    krl_status ls = level_const(g, d, L);
    if (ls != KRL_OK) return ls;
    ls = level_scratch(g);
    if (ls != KRL_OK) return ls;
    const int ncell = g->ncell;
    const size_t n = (size_t)ncell;
    if (init_lte) KRL_CUDA(levels_lte(L, d->n_mol, ncell, pops, s), "levels lte");
    KRL_CUDA(cudaMemcpyAsync(g->lv_pops0, pops, n * L.n * sizeof(double), cudaMemcpyDeviceToDevice, s), "levels");
    for (int it = 0; it < n_iter; ++it) {
        for (int t = 0; t < L.n_trans; ++t) {
            const int u = L.tu[t], l = L.tl[t];
            KRL_CUDA(levels_field(pops, ncell, L.n, l, 1.0, g->opacity, s), "lower-level field");
            KRL_CUDA(levels_field(g->lv_pops0, ncell, L.n, u, L.A[u][l], g->lv_rate, s), "frozen emission");
            KRL_CUDA(levels_sum_rate(g->lv_pops0, ncell, L.n, u, L.A[u][l], g->lv_total, s), "emission total");
            krl_line_desc ld{};
            ld.nu0_hz = (L.E[u] - L.E[l]) * kKB / kHPlanck;
            ld.mass_amu = d->mass_amu;
            ld.A_ul = L.A[u][l];
            ld.g_u = L.g[u];
            ld.g_l = L.g[l];
            ld.k_ul = L.k[u][l];
            ld.src_kind = KRL_SRC_VOLUME;
            ld.src_profile = KRL_PROFILE_GAUSSIAN;
            ld.src_rate = g->lv_rate;
            ld.band_axis = -1;
            ld.luminosity = 1.0;
            ld.spec_xmin = -40.0;
            ld.spec_xmax = 40.0;
            ld.spec_nbins = 80;
            ld.tally_flags = KRL_TALLY_EXC;
            krl_status rs = krl_line_set(g, &ld, st);
            if (rs != KRL_OK) return rs;
            const uint64_t first = ((uint64_t)it * L.n_trans + t) * packets_per_line;
            rs = krl_run_packets(g, packets_per_line, first, seed, nullptr, nullptr, nullptr, st);
            if (rs != KRL_OK) return rs;
            KRL_CUDA(levels_gamma(g->exc, ncell, g->lv_total, g->cell_cm, g->info.sigma0_cm2, (double)packets_per_line,
                                  g->lv_gamma + (size_t)t * n, s),
                     "gamma");
        }
        KRL_CUDA(cudaMemsetAsync(g->lv_change, 0, sizeof(unsigned long long), s), "levels");
        KRL_CUDA(levels_solve(L, g->lv_gamma, ncell, g->n_coll, d->n_mol, pops, g->lv_change, s), "levels solve");
        if (max_change) {
            unsigned long long bits = 0;
            KRL_CUDA(cudaMemcpyAsync(&bits, g->lv_change, 8, cudaMemcpyDeviceToHost, s), "levels");
            KRL_CUDA(cudaStreamSynchronize(s), "levels");
            memcpy(max_change + it, &bits, 8);
        }
    }
    return KRL_OK;
}

size_t krl_tally_bytes(const krl_grid* g, krl_tally_kind kind)
{
    if (!g || !g->line_ok) return 0;
    size_t esz;
    size_t n = tally_elems(g, kind, &esz);
    return n * esz;
}

krl_status krl_tallies_get(krl_grid* g, krl_tally_kind kind, void* dst, size_t bytes, krl_stream st)
{
    if (!g || !dst) return fail(KRL_ERR_ARG, "krl_tallies_get: NULL argument");
    if (!g->line_ok) return fail(KRL_ERR_STATE, "no line set");
    size_t esz;
    size_t n = tally_elems(g, kind, &esz);
    if (n == 0) return fail(KRL_ERR_ARG, "tally %d is not enabled", (int)kind);
    if (bytes != n * esz) return fail(KRL_ERR_ARG, "tally %d needs %zu bytes, got %zu", (int)kind, n * esz, bytes);
    KRL_CUDA(cudaMemcpyAsync(dst, tally_ptr(g, kind), bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)st),
             "krl_tallies_get");
    return KRL_OK;
}

krl_status krl_tallies_reset(krl_grid* g, krl_stream st)
{
    if (!g) return fail(KRL_ERR_ARG, "krl_tallies_reset: NULL grid");
    if (!g->line_ok) return fail(KRL_ERR_STATE, "no line set");
    return zero_tallies(g, (cudaStream_t)st);
}

}  // extern "C"
