// Internal declarations shared by the CUDA translation units of libkrl.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "krl.h"

namespace krl {

// ---------------------------------------------------------------- table geometry
// ph_mode 2 Voigt slice: nodes uniform in log10|x| on [-4, 3] (Sec. 2.2.1, 2.3.1).
constexpr int kVoigtN = 5000;
constexpr double kVoigtL0 = -4.0;
constexpr double kVoigtL1 = 3.0;
// Velocity sampler (Sec. 2.1.1): 40 incoming-frequency rows, 251 u-nodes.
constexpr int kUsNx = 40;
constexpr int kUsNu = 251;
constexpr double kUsU0 = -6.0;
constexpr double kUsDu = 0.048;
constexpr double kUsFloor = 1e-30;
// R_IIA table (Eq. riia-table): Delta x |x_in| x g.
constexpr int kRnD = 201;
constexpr int kRnX = 200;
constexpr int kRnG = 40;
constexpr double kRdMax = 10.0;
constexpr double kRdStep = 0.1;
constexpr double kRxMax = 120.0;
constexpr double kRsMin = 0.1;
constexpr size_t kRtabElems = (size_t)kRnG * kRnX * kRnD;
// The R table regrouped by interpolation cell: entry (k, j, i) holds the four
// corners (g_k, x_j), (g_k, x_j+1), (g_k+1, x_j), (g_k+1, x_j+1) at Delta_i,
// so a trilinear lookup reads two float4 instead of eight floats.
constexpr size_t kRquadElems = (size_t)(kRnG - 1) * (kRnX - 1) * kRnD;

// Search guide of the sampler rows: for each row, kGuideN bins uniform in
// logit(xi) = ln(xi / (1 - xi)) on [-kGuideW, kGuideW]; entry m is the
// largest node j whose CDF is <= sigmoid(left edge of bin m). A lookup starts
// there and walks to the exact node, so the guide only shortens the search.
constexpr int kGuideN = 256;
constexpr double kGuideW = 16.7;

// Row guide of the sampler: bins of |x| by the top bits of its float32
// encoding (exponent and 4 mantissa bits: 16 bins per octave) from 0.25 up
// to 512; entry t is the largest row i <= kUsNx - 2 whose node x_i is <= the
// bin's lower edge. Every bin holds at most one node (the rows are 4/9 apart
// below |x| = 8 and a factor 1.19 apart above; a CPU test checks the node
// set), so the row of any |x| is the entry or the one after it.
constexpr int kRowGuideN = 176;
constexpr unsigned kRowGuideBase = 0x3E800000u >> 19;   // float32 bits of 0.25, >> 19

// Shared-memory image of the per-line sampling tables used by the walk.
constexpr int kSmemVoigt = 0;
constexpr int kSmemUsX = kVoigtN;                 // 40 floats
constexpr int kSmemUsC = kVoigtN + 48;            // 40 x 251 floats
constexpr int kSmemFloats = kSmemUsC + kUsNx * kUsNu;
constexpr int kSmemGuideBytes = kUsNx * kGuideN;  // uint8 after the floats
constexpr int kSmemRowGuide = kSmemFloats * (int)sizeof(float) + kSmemGuideBytes;   // byte offset
constexpr size_t kSmemBytes = (size_t)kSmemRowGuide + 192;

// ---------------------------------------------------------------- compile-time walk features
enum : unsigned {
    F_VEL = 1u,       // cells carry a bulk velocity
    F_SCAT = 2u,      // per-cell scattering counts
    F_RICH = 4u,      // excitation / mean intensity / emissivity / destruction
};

enum { ST_EMITTED = 0, ST_ESCAPED, ST_DESTROYED, ST_STUCK, ST_SCAT, ST_CROSS, ST_ABSORBED, ST_N = 8 };

// A packet whose weight falls below this after continuum absorption ends.
constexpr double kWeightCut = 1e-12;

// Philox4x32-10 round keys of a launch: k[0][r] = key_lo + r 0x9E3779B9,
// k[1][r] = key_hi + r 0xBB67AE85 (mod 2^32). Precomputed on the host and
// passed in the kernel's parameter block, so each round reads its keys as
// constant operands instead of recomputing the schedule per call.
struct RoundKeys {
    unsigned k[2][10];
};

inline RoundKeys round_keys(unsigned long long seed)
{
    RoundKeys K;
    unsigned k0 = (unsigned)(seed & 0xffffffffu), k1 = (unsigned)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k[0][r] = k0;
        K.k[1][r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}

struct TransportArgs {
    const float4* cells;      // {line-centre tau per cell width, Vx/b, Vy/b, Vz/b}
    const float* eps;         // per-cell destruction probability or nullptr
    const float* tau_abs;     // per-cell continuum absorption per cell width or nullptr
    double* absw;             // [ncell] absorbed weight (with tau_abs)
    int nx, ny, nz, ncell;
    unsigned periodic;        // bit d set: axis d periodic
    double a;                 // damping parameter (the FP32 walk rounds it once)
    const float* H0;          // device scalar H(a, 0)
    const float* voigt_lnH;
    const float* us_x;
    const float* us_lncdf;
    const unsigned char* us_guide;
    const float* rtab;
    const float4* rquad;      // rtab by interpolation cell (the deposit's second stage)
    int src_kind, src_profile, src_axis, band_axis;
    double src_pos[3];
    double src_plane, band_lo, band_hi;
    const double* src_cdf;
    double spec_lo, spec_hi;
    int spec_n;
    int n_ch;
    double ch_x0, ch_dx;      // v_min / b, dv / b (the FP32 walk rounds them once)
    int n_cam;
    float cam[KRL_MAX_CAMERAS][3];
    unsigned rich;            // KRL_TALLY_EXC | KRL_TALLY_J | KRL_TALLY_EMISS, eps present (bit 16)
    double* spec_w;
    unsigned long long* spec_c;
    unsigned long long* scat;
    double* exc;
    double* J;
    float* emiss;
    unsigned long long* stats;   // [ST_N] for this launch
    unsigned long long* next;    // work counter, zero at launch
    krl_packet_record* rec;
    unsigned long long first, n;
    unsigned k0, k1;
    RoundKeys keys;           // round keys of (k0, k1)
    unsigned long long max_iters;
    unsigned max_iters32;     // min(max_iters, 2^32 - 1): the per-event check in 32 bits
    int refill_min;
    // line-profile mode (krl_line_desc.ph_mode: 2, or 1 / 3 below)
    int ph_mode;
    const float* voigt2d;     // [kV2Na][kV2Nx] ln H, mode 1
    int v2_row;               // mode 1: rows v2_row, v2_row + 1 bracket log10 a
    double v2_w;              // mode 1: weight of row v2_row + 1
    double u0;                // mode 3: core-wing crossing point
    // two-stage emissivity deposit (FP32 walk): segment records, 2 float4
    // each ({cell bits, base, x_com, nx}, {ny, nz, 0, 0}); count may run past
    // the capacity (the segments beyond it are deposited by the walk)
    float4* seg;
    unsigned long long* seg_count;
    unsigned long long seg_cap;
};

constexpr unsigned kRichEps = 1u << 16;

// Two-dimensional Voigt table of line-profile mode 1: ln H(a_j, x_i), a_j
// uniform in log10 a on [kV2LaMin, kV2LaMax], x_i uniform in log10|x| on
// [kVoigtL0, kVoigtL1].
constexpr int kV2Na = 64;
constexpr int kV2Nx = 512;
constexpr double kV2LaMin = -6.0;
constexpr double kV2LaMax = 0.0;
// work: at least 64 doubles of device scratch.
cudaError_t build_voigt2d(float* out, double* work, cudaStream_t s);

// Launch the walk (transport.cu). grid/block chosen by the caller.
cudaError_t launch_transport(const TransportArgs& A, int precision, unsigned features,
                             int grid, int block, cudaStream_t s);
// Second stage of the emissivity deposit over the records A.seg[0 ..
// min(*A.seg_count, A.seg_cap)), on the stream after the walk that wrote them.
cudaError_t launch_emiss_deposit(const TransportArgs& A, unsigned features, int sm_count, cudaStream_t s);
// Many models in one launch: models[m] holds model m's full argument block
// (its own work counter `next`, run counters `stats`, tables and tallies).
struct BatchArgs {
    const TransportArgs* models;   // device [n_models]
    int n_models;
    int* cursor;                   // device: lowest model that may still have work
    RoundKeys keys;                // one seed for every model of the batch
};
cudaError_t launch_transport_batch(const BatchArgs& B, int precision, unsigned features, int grid, int block,
                                   cudaStream_t s);

// Occupancy of one instantiation (CTAs per SM at this block size).
int transport_occupancy(int precision, unsigned features, int block, int ph_mode = 2);
// Line-profile modes 1 and 3 (transport_modes.cu).
cudaError_t launch_transport_ph(const TransportArgs& A, int ph_mode, int precision, unsigned features, int grid,
                                int block, cudaStream_t s);
int transport_occupancy_ph(int ph_mode, int precision, unsigned features, int block);
// Largest CTA the instantiation is compiled for (512 lean FP32, else 256).
int transport_max_block(int precision, unsigned features);
// The batched launch: its CTA size limit and occupancy.
int transport_batch_max_block();
int transport_batch_occupancy(int precision, unsigned features, int block);

// ---------------------------------------------------------------- ray trace (raytrace.cu)
struct RayArgs {
    const float4* cells;      // per-cell record (alpha0 dx, V/b)
    const float* tau_abs;     // continuum absorption per cell width, or nullptr
    int nx, ny, nz;
    const float* voigt_lnH;
    const float* H0;
    float a;
    const float* emiss;       // [ncell][n_ch] camera-directed scattering emissivity
    const float* jline;       // [ncell] frequency-integrated line emission, or nullptr
    float* hcube;             // [ncell][n_ch] scratch for the per-camera profile, or nullptr
                              // (then the trace evaluates the profile per segment)
    float4* rayinit;          // with hcube: [npix][2] scratch for each ray's start
                              // ({cell x, y, z, hit} as ints, {in-cell x, y, z, -})
    int n_ch;
    double ch_x0, ch_dx;      // v_min / b, dv / b
    double n[3], u[3], v[3];  // camera direction and image axes
    float dirf[3];            // the march direction -n in float
    float face_neg[3], face_c[3];   // distance to the face ahead on axis d from in-cell
                                    // position p: fma(p, face_neg[d], face_c[d])
    double centre[3];         // image centre (box centre), cell units
    double pix;               // pixel size, cell units
    int npix_x, npix_y;
    float* maps;              // [n_ch][npix_y][npix_x]
};
cudaError_t launch_raytrace(const RayArgs& A, int sm_count, cudaStream_t s);

// ---------------------------------------------------------------- statistical equilibrium (levels.cu)
constexpr int kMaxLevels = KRL_MAX_LEVELS;
constexpr int kMaxTrans = kMaxLevels * (kMaxLevels - 1) / 2;
struct LevelConst {
    int n;                              // levels
    double T;                           // gas temperature [K]
    double E[kMaxLevels];               // energies / k_B [K]
    double g[kMaxLevels];
    double A[kMaxLevels][kMaxLevels];   // A[u][l], u > l
    double k[kMaxLevels][kMaxLevels];   // k_coll[u][l], u > l
    int n_trans;                        // radiative pairs, ordered by (l, u)
    int tu[kMaxTrans], tl[kMaxTrans];
};
cudaError_t levels_lte(const LevelConst& L, const float* n_mol, int ncell, double* pops, cudaStream_t s);
cudaError_t levels_field(const double* pops, int ncell, int n_lev, int lev, double scale, float* out, cudaStream_t s);
// total: device scratch of levels_sum_scratch_doubles() doubles; the sum lands in total[0].
size_t levels_sum_scratch_doubles();
cudaError_t levels_sum_rate(const double* pops, int ncell, int n_lev, int u, double A, double* total, cudaStream_t s);
cudaError_t levels_gamma(const double* exc, int ncell, const double* total, double dx, double sigma0, double n_packets,
                         double* gamma, cudaStream_t s);
cudaError_t levels_solve(const LevelConst& L, const double* gamma, int ncell, const float* n_coll, const float* n_mol,
                         double* pops, unsigned long long* max_change, cudaStream_t s);

// ---------------------------------------------------------------- setup kernels (tables.cu)
struct LineTables {
    float* voigt_lnH;   // [kVoigtN]
    float* H0;          // [1]
    float* us_x;        // [kUsNx]
    float* us_lncdf;    // [kUsNx * kUsNu]
    unsigned char* us_guide;  // [kUsNx * kGuideN]
    float* rtab;        // [kRtabElems]
    float4* rquad;      // [kRquadElems] (built with rtab)
    double* work;       // scratch: Weideman coefficients + R-table masses
};
size_t line_tables_work_doubles();
cudaError_t build_line_tables(double a, const LineTables& T, bool with_r, cudaStream_t s);

struct FieldArgs {
    int ncell;
    int opacity_kind;
    const float* opacity;
    const float* vx;
    const float* vy;
    const float* vz;
    const float* n_coll;
    double tau_scale;     // sigma0 * cell_cm for KRL_OPACITY_NL, 1 for TAU
    double inv_b;
    double k_ul, A_ul;
    float4* cells;
    float* eps;           // may be nullptr
};
cudaError_t derive_fields(const FieldArgs& F, cudaStream_t s);

// Flags bad values (NaN, Inf, negative where forbidden) into *bad (int, device).
cudaError_t validate_field(const float* f, int n, bool allow_negative, int* bad, cudaStream_t s);

// Inclusive FP64 scan of rate[n] (float), normalised by its last element.
cudaError_t emission_cdf(const float* rate, int n, double* cdf, double* work, size_t work_doubles,
                         int* bad, cudaStream_t s);
size_t emission_cdf_work_doubles(int n);

// dst[m][k] += src[m * ST_N + k] for m < n_models, k < ST_N (64-bit counters).
cudaError_t add_counters_batch(unsigned long long* const* dst, const unsigned long long* src, int n_models,
                               cudaStream_t s);

// out[i] += in[i], 64-bit counters.
cudaError_t add_counters(unsigned long long* out, const unsigned long long* in, int n, cudaStream_t s);

}  // namespace krl
