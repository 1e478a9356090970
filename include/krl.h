/*
 * krl.h - C ABI of the GB300 Monte Carlo line-transfer library (libkrl.so).
 *
 * The library implements the Monte Carlo photon-packet pass of the
 * Kratos-linerad method (arXiv 2608.09340, Sec. 2): per-packet random walks
 * through a 3-D Cartesian grid with optical-depth integration against a
 * Voigt profile in the comoving frame (Sec. 2.1, Eq. xdef, Eq. sigma0),
 * angle-dependent partial redistribution sampled from tables (Sec. 2.1.1,
 * 2.1.2, Eq. riia-scatter), and tallies of the escaped spectrum, the
 * excitation rate (Sec. 2.1.3), the velocity-resolved mean intensity and the
 * camera-directed scattering emissivity (Sec. 2.2.1, Eq. scat-line); the
 * three line-profile modes (Sec. 2.3.1) and continuum absorption (Sec. 3.2)
 * in that pass; many models in one persistent launch (krl_batch_*); the
 * channel-map ray trace of the two-step imaging (Sec. 2.2.2,
 * krl_raytrace_channels); statistical equilibrium and the Lambda iteration
 * (Sec. 2.1.3, krl_levels_*).
 *
 * Conventions shared by every call:
 *  - Pointers documented as "device" are CUDA device pointers (for example
 *    torch.Tensor.data_ptr()); "host" pointers are ordinary CPU memory.
 *  - Caller buffers are BORROWED for the duration of the call only; the
 *    library copies what it keeps. The library owns everything it allocates
 *    and frees it in krl_grid_destroy.
 *  - Every call is ordered on the caller's stream `s` (a cudaStream_t; NULL
 *    is the legacy default stream). A call synchronises `s` only when it
 *    returns host data (documented per call).
 *  - Every call returns a krl_status; on failure krl_last_error() returns a
 *    thread-local message. No C++ exception crosses this boundary.
 *  - Frequencies are in Doppler units x = (nu - nu0) / nu_D, positive to the
 *    blue; a velocity v along the line of sight (receding positive) maps to
 *    x = -v / b. Lengths inside the library are in cell widths.
 *  - Grid fields are float32, C order [nz][ny][nx] (x fastest).
 */
#ifndef KRL_H
#define KRL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define KRL_API __attribute__((visibility("default")))
#else
#define KRL_API
#endif

typedef struct CUstream_st* krl_stream;

typedef enum {
    KRL_OK = 0,
    KRL_ERR_ARG = -1,      /* invalid argument; nothing was enqueued            */
    KRL_ERR_CUDA = -2,     /* a CUDA runtime call failed                         */
    KRL_ERR_OOM = -3,      /* device allocation failed                           */
    KRL_ERR_BUDGET = -4,   /* some packets hit the per-packet iteration budget   */
    KRL_ERR_STATE = -5,    /* call out of order (e.g. run before krl_line_set)   */
    KRL_ERR_NUMERIC = -6   /* NaN / negative field value, or a device numeric fault */
} krl_status;

/* Thread-local description of the last failure on this thread. */
KRL_API const char* krl_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
KRL_API int krl_version(void);

/* ------------------------------------------------------------------ grid */

enum { KRL_PERIODIC_X = 1u, KRL_PERIODIC_Y = 2u, KRL_PERIODIC_Z = 4u };

/* How `opacity` is given. */
enum {
    KRL_OPACITY_TAU = 0,   /* line-centre optical depth per cell width, n_l sigma0 dx */
    KRL_OPACITY_NL = 1     /* lower-level number density n_l [cm^-3] (Eq. sigma0)     */
};

typedef struct {
    int nx, ny, nz;             /* cells per axis, each >= 1; nx*ny*nz < 2^31     */
    double cell_cm;             /* cubic cell width [cm], > 0                      */
    uint32_t boundary_flags;    /* KRL_PERIODIC_*; other faces are open (escape)   */
    int opacity_kind;           /* KRL_OPACITY_TAU or KRL_OPACITY_NL               */
    const float* opacity;       /* device [nz][ny][nx], >= 0, required             */
    double T_K;                 /* gas temperature [K], uniform (a single b and a
                                   per line, the ph_mode 2 setting of Sec. 2.2.1)  */
    const float* vx;            /* device [nz][ny][nx] bulk velocity [cm/s] or NULL */
    const float* vy;
    const float* vz;
    const float* n_coll;        /* device collider density [cm^-3] or NULL (Eq. eps) */
    const float* tau_abs;       /* device continuum (dust) absorption optical depth per
                                   cell width, >= 0, or NULL. The packet weight decays
                                   as exp(-tau_abs ds) along each segment and the
                                   segment's tallies take the mean weight
                                   (1 - exp(-dtau))/dtau (Eq. scat-line); the ray
                                   trace adds it to the line opacity. A packet whose
                                   weight falls below 1e-12 ends as absorbed.      */
} krl_grid_desc;

typedef struct krl_grid krl_grid;

/*
 * Create a grid: validates the fields (KRL_ERR_NUMERIC on NaN, Inf or a
 * negative opacity / density) and copies them into library-owned device
 * memory. Synchronises `s` (for the validation result). The fields are
 * borrowed for this call only.
 */
KRL_API krl_status krl_grid_create(krl_grid** out, const krl_grid_desc* desc, krl_stream s);

/* Free everything the grid owns. Synchronises the device. NULL is a no-op. */
KRL_API krl_status krl_grid_destroy(krl_grid* g);

/* ------------------------------------------------------------------ line */

enum { KRL_SRC_POINT = 0, KRL_SRC_PLANE = 1, KRL_SRC_BEAM = 2, KRL_SRC_VOLUME = 3 };
enum { KRL_PROFILE_LINE_CENTRE = 0, KRL_PROFILE_GAUSSIAN = 1 };
enum { KRL_TALLY_SCATMAP = 1u, KRL_TALLY_EXC = 2u, KRL_TALLY_J = 4u, KRL_TALLY_EMISS = 8u };
#define KRL_MAX_CAMERAS 8

typedef struct {
    /* two-level line (Sec. 2.1) */
    double nu0_hz;              /* rest frequency                                   */
    double mass_amu;            /* mass of the absorber                             */
    double A_ul;                /* Einstein A [s^-1]                                */
    double g_u, g_l;            /* degeneracies                                     */
    double k_ul;                /* collisional de-excitation coefficient [cm^3/s];
                                   with the grid's n_coll gives epsilon (Eq. eps)  */
    double a_fixed;             /* > 0: damping parameter; else A_ul/(4 pi nu_D)    */
    /* photon source (Sec. 3) */
    int src_kind;               /* KRL_SRC_*                                        */
    double src_pos[3];          /* POINT: position (x, y, z) in cell units           */
    int src_axis;               /* PLANE: normal axis; BEAM: travel axis (+ sense)  */
    double src_plane;           /* PLANE: coordinate along src_axis, cell units      */
    int band_axis;              /* BEAM: transverse axis with a limited entry band,
                                   -1 for the whole face                            */
    double band_lo, band_hi;    /* BEAM: band [lo, hi) in cell units                 */
    int src_profile;            /* KRL_PROFILE_LINE_CENTRE or KRL_PROFILE_GAUSSIAN
                                   (thermal profile exp(-x^2)/sqrt(pi))            */
    const float* src_rate;      /* VOLUME: device per-cell emission weight (>= 0)   */
    double luminosity;          /* photons per second of the whole run (scales
                                   physical outputs; raw tallies use unit weight)  */
    /* escaped spectrum (lab frame, all directions) */
    double spec_xmin, spec_xmax;
    int spec_nbins;             /* >= 1; bins half-open, plus under/overflow        */
    /* velocity channels v_k = v_min + (k + 1/2) dv (Sec. 2.2.1) */
    double ch_vmin_cms, ch_dv_cms;
    int n_ch;                   /* 0 when neither J nor the emissivity is tallied   */
    /* cameras: unit propagation direction toward the camera
       (sin t cos p, sin t sin p, cos t) */
    int n_cam;
    double cam_theta[KRL_MAX_CAMERAS], cam_phi[KRL_MAX_CAMERAS];
    uint32_t tally_flags;       /* KRL_TALLY_*                                      */
    /* line-profile mode (Sec. 2.3.1); the velocity sampler is the same in all:
       0 or 2: the Voigt slice at this a, tables in shared memory (production);
       1: H(a, x) from a two-dimensional table of ln H over 64 damping parameters
          (log10 a uniform on [-6, 0]) by 512 frequencies (log10|x| uniform on
          [-4, 3]) in global memory, bilinear in (log10 a, log10|x|), and the
          sampler read from global memory; needs 1e-6 <= a <= 1;
       3: the core-wing approximation (1 - w) exp(-x^2) + w a / (sqrt(pi)(x^2 +
          a^2)), w = [1 + tanh(2|x| - 2 u0)] / 2, u0 the outer crossing point of
          the two terms; it shows what an inconsistent profile costs and is unsuited
          to production runs; needs a < 0.8.
       Modes 1 and 3 run krl_run_packets only (KRL_ERR_ARG from krl_batch_run
       and krl_raytrace_channels, which use the mode 2 slice).                 */
    int ph_mode;
} krl_line_desc;

/*
 * Attach a line to the grid: derives b = (2kT/m)^{1/2}, nu_D, a, sigma0
 * (Eq. sigma0) and epsilon (Eq. eps); builds, in FP64 on the device, the
 * ph_mode 2 Voigt slice at this a (5000 nodes in log10|x| on [-4, 3]), the
 * velocity sampler (40 x-nodes x 251 u-nodes, log CDF) and the R_IIA table
 * (Eq. riia-table, 201 Delta x 200 |x| x 40 g) and stores them as float32;
 * derives the per-cell record {alpha0 dx, V/b}; allocates and zeroes the
 * tallies. Replaces any previous line. Enqueued on `s`, which it
 * synchronises once at the end (to read H(a,0) and the source-rate check:
 * KRL_ERR_NUMERIC for a NaN/negative rate, KRL_ERR_ARG for a zero total).
 */
KRL_API krl_status krl_line_set(krl_grid* g, const krl_line_desc* d, krl_stream s);

typedef struct {
    double b_cms, nu_D_hz, a, sigma0_cm2, H0;  /* H0 = H(a, 0) as stored */
    int ncell;
} krl_line_info;

/* Derived line constants (host). */
KRL_API krl_status krl_line_info_get(const krl_grid* g, krl_line_info* out);

/* ------------------------------------------------------------------ packets */

enum { KRL_PREC_FP32 = 0, KRL_PREC_FP64 = 1 };

/* Launch tuning; pass NULL for the defaults. Zero fields take the default. */
typedef struct {
    int precision;              /* KRL_PREC_FP32 (production) or KRL_PREC_FP64
                                   (same walk in double, for lockstep checks)       */
    int block;                  /* threads per CTA, multiple of 32; at most 512 for
                                   the FP32 walk without rich tallies (its default),
                                   256 otherwise (the default there)               */
    int ctas_per_sm;            /* resident CTAs per SM of the persistent grid      */
    int refill_min;             /* a warp takes new packets once at least this many
                                   of its lanes are idle (1..32)                    */
    uint64_t max_iters;         /* per-packet cap on walk iterations (budget);
                                   0: 2^32 - 1 (the default); larger values are
                                   rejected with KRL_ERR_ARG (the walk counts a
                                   packet's events in 32 bits)                      */
    int64_t emiss_records;      /* FP32 runs with an emissivity tally deposit it in
                                   two stages: the walk records each segment (32 B)
                                   in a stream-ordered buffer of this many records,
                                   then one warp per segment adds its channels.
                                   0: 64 per packet, clamped to [2^16, 2^25];
                                   -1: deposit inside the walk (no buffer); at most
                                   2^36 (KRL_ERR_ARG beyond). Segments
                                   beyond the buffer, and every segment when it
                                   cannot be allocated, are deposited by the walk:
                                   the result is the same up to the order of the
                                   FP32 atomic additions                            */
    int table_space;            /* where the FP32 walk of profile mode 2 reads the
                                   Voigt slice and the sampler's nodes and ln CDF:
                                   KRL_TABLES_SHARED (0, default): staged into
                                   shared memory per CTA; KRL_TABLES_CONSTANT (1):
                                   the constant bank, the placement Sec. 2.3.1
                                   recommends (copied in before the launch; runs
                                   with it must not overlap on the device). For
                                   measurement; KRL_ERR_ARG for other modes and
                                   for the FP64 walk                               */
} krl_tune;

enum { KRL_TABLES_SHARED = 0, KRL_TABLES_CONSTANT = 1 };

/* One record per packet of a run (optional output). */
typedef struct {
    float x;                    /* lab-frame x at escape / destruction             */
    uint32_t nscat;             /* scatterings                                     */
    uint32_t ncross;            /* cell-face crossings                             */
    uint16_t status;            /* 1 escaped, 2 destroyed, 3 budget exhausted,
                                   4 absorbed (weight below the cut)                */
    uint16_t pad;
    uint32_t cell0;             /* flat index of the emission cell                 */
    uint32_t scat_cells;        /* FP64 walk: sum over the packet's scatterings of
                                   the flat index of the cell it scattered in
                                   (mod 2^32), a check that two walks scattered in
                                   the same cells; 0 from the FP32 walk            */
} krl_packet_record;

typedef struct {
    uint64_t emitted, escaped, destroyed, stuck, scatterings, crossings;
    uint64_t absorbed;          /* packets whose weight fell below the cut          */
} krl_run_stats;

/*
 * Run packets with ids [first_id, first_id + n) under key `seed`
 * (Philox4x32-10, counter = (id, event, block)) and ACCUMULATE into the
 * grid's tallies. Each packet's random stream depends only on (seed, id),
 * never on the launch shape. records (device, may be NULL) receives
 * records[id - first_id]. stats (host, may be NULL): when given, the call
 * synchronises `s` and returns this run's counters, and returns
 * KRL_ERR_BUDGET if any packet exhausted max_iters. n = 0 is a no-op.
 * Runs of one grid may be in flight at once on different streams and be
 * issued from several host threads: each takes the next of 8 scratch slots
 * in turn, and a run that reuses a slot first waits, on its own stream, for
 * the slot's previous run to finish with it (an event recorded after that
 * run's last read of the slot); tallies accumulate atomically, so their
 * order does not matter beyond FP64 rounding. A run enqueued while `s` is
 * being captured into a CUDA graph keeps its slot inside the graph without
 * that wait: replays of such a graph must not overlap other runs of the grid.
 * An FP32 run of a line with an emissivity tally also allocates and frees
 * its segment buffer in stream order on `s` (cudaMallocAsync / cudaFreeAsync,
 * size set by krl_tune.emiss_records), so the call stays capturable in a
 * CUDA graph; the buffer is the run's own and never outlives it.
 */
KRL_API krl_status krl_run_packets(krl_grid* g, uint64_t n, uint64_t first_id, uint64_t seed,
                           const krl_tune* tune, krl_packet_record* records,
                           krl_run_stats* stats, krl_stream s);

/* ------------------------------------------------------------------ tallies */

typedef enum {
    KRL_OUT_SPEC_W = 0,   /* double [spec_nbins + 2]: under, bins, over (escaped
                             packet weights)                                       */
    KRL_OUT_SPEC_N = 1,   /* uint64 [spec_nbins + 2]: packet counts               */
    KRL_OUT_SCATMAP = 2,  /* uint64 [ncell]: scatterings per cell                  */
    KRL_OUT_EXC = 3,      /* double [ncell]: sum of w ds H(a, x_com) (ds in cells)  */
    KRL_OUT_J = 4,        /* double [ncell][n_ch]: sum of w ds per comoving channel */
    KRL_OUT_EMISS = 5,    /* float [n_cam][ncell][n_ch]: sum of
                             w ds alpha0 H(a,x_in) R(x_out,k; x_in, g) / 4 pi      */
    KRL_OUT_STATS = 6,    /* uint64 [8]: emitted, escaped, destroyed, stuck,
                             scatterings, crossings, absorbed, 0 (all runs since
                             reset)                                                */
    KRL_OUT_ABSW = 7,     /* double [ncell]: packet weight absorbed by the continuum
                             (grids with tau_abs)                                  */
    /* read-only views of what krl_line_set built (float32 unless noted) */
    KRL_OUT_VOIGT = 16,   /* [5000]: ln H(a, 10^l), l = -4 + 7 i / 4999           */
    KRL_OUT_US_X = 17,    /* [40]: sampler incoming-frequency nodes |x|           */
    KRL_OUT_US_LNCDF = 18,/* [40][251]: ln CDF of u_par at u_j = -6 + 0.048 j       */
    KRL_OUT_RTAB = 19,    /* [40 g][200 |x|][201 Delta] R_IIA table (emissivity only) */
    KRL_OUT_CELLS = 20,   /* float4 [ncell]: {alpha0 dx, Vx/b, Vy/b, Vz/b}         */
    KRL_OUT_EPS = 21,     /* [ncell]: destruction probability (when k_ul, n_coll)  */
    KRL_OUT_SRC_CDF = 22, /* double [ncell]: emission CDF (volume source)         */
    KRL_OUT_H0 = 23,      /* [1]: H(a, 0)                                          */
    KRL_OUT_VOIGT2D = 24  /* [64][512]: ln H of ph_mode 1 (built on its first use)  */
} krl_tally_kind;

/*
 * Copy one accumulated tally (raw, unit packet weight, code units), or one
 * of the line's tables / per-cell records, into the caller's device buffer
 * dst (bytes must equal the output's size, see krl_tally_bytes).
 * Enqueued on `s`; does not synchronise.
 */
KRL_API krl_status krl_tallies_get(krl_grid* g, krl_tally_kind kind, void* dst, size_t bytes,
                           krl_stream s);

/* Size in bytes of a tally (0 if it is not enabled). */
KRL_API size_t krl_tally_bytes(const krl_grid* g, krl_tally_kind kind);

/* Zero all tallies and counters. Enqueued on `s`. */
KRL_API krl_status krl_tallies_reset(krl_grid* g, krl_stream s);

/* ------------------------------------------------------------------ level populations */

#define KRL_MAX_LEVELS 8

typedef struct {
    int n_lev;                                       /* 2 .. KRL_MAX_LEVELS             */
    double E_K[KRL_MAX_LEVELS];                      /* level energies / k_B [K]        */
    double g[KRL_MAX_LEVELS];                        /* degeneracies                    */
    double A[KRL_MAX_LEVELS][KRL_MAX_LEVELS];        /* A[u][l] (u > l) [s^-1]; > 0
                                                        marks a radiative line          */
    double k_coll[KRL_MAX_LEVELS][KRL_MAX_LEVELS];   /* k[u][l] (u > l) collisional
                                                        de-excitation [cm^3 s^-1]       */
    double mass_amu;
    const float* n_mol;                              /* device [ncell] molecule density */
} krl_levels_desc;

/*
 * Statistical equilibrium per cell (Sec. 2.1.3; Eq. boltzmann generalised
 * to n levels), FP64, one thread per cell: collisions k_ul n_coll (the
 * grid's n_coll field) and their detailed-balance inverses at the grid's T,
 * radiative pumping Gamma_lu and spontaneous plus stimulated emission
 * A_ul + (g_l/g_u) Gamma_lu, sum of populations = n_mol. gamma: device
 * double [n_trans][ncell], the radiative pairs ordered by lower then upper
 * level. pops: device double [ncell][n_lev], written. max_change (host, may
 * be NULL): max over cells and levels of |n_new - n_old| / n_mol against the
 * values pops held on entry; when given, the call synchronises `s`.
 */
KRL_API krl_status krl_levels_solve(krl_grid* g, const krl_levels_desc* d, const double* gamma, double* pops,
                                    double* max_change, krl_stream s);

/*
 * Lambda iteration (Sec. 2.1.3). init_lte != 0: pops starts from
 * collisional equilibrium (Boltzmann at the grid's T); otherwise from the
 * values in pops. The emission of every radiative line is frozen at the
 * starting populations (volume source n_u A_ul, thermal profile). Each of
 * n_iter cycles, for every line: sets the grid's opacity field to the
 * current lower-level population, attaches the line (krl_line_set: its own
 * b, a, sigma0, epsilon, tables), runs packets_per_line packets (ids
 * distinct per cycle and line, key `seed`), turns the excitation tally into
 * Gamma; then solves the populations (krl_levels_solve). The grid must have
 * been created with KRL_OPACITY_NL; its opacity field and line are left as
 * the last cycle set them. max_change (host [n_iter] or NULL) receives each
 * cycle's change; the call synchronises `s` once per line and cycle.
 */
KRL_API krl_status krl_levels_iterate(krl_grid* g, const krl_levels_desc* d, int n_iter, uint64_t packets_per_line,
                                      uint64_t seed, int init_lte, double* pops, double* max_change, krl_stream s);

/* ------------------------------------------------------------------ batched models */

typedef struct krl_batch krl_batch;

/*
 * A set of grids (independent models, each with its own line and tables)
 * to be run together by krl_batch_run. Uploads nothing yet; synchronises
 * `s`. The grids must live on the current device and stay alive, and their
 * lines must not change (krl_batch_run checks) while the batch is used.
 */
KRL_API krl_status krl_batch_create(krl_batch** out, krl_grid* const* grids, int n_models, krl_stream s);
KRL_API krl_status krl_batch_destroy(krl_batch* b);

/*
 * Run packets[m] packets with ids [first_ids[m], first_ids[m] + packets[m])
 * (first_ids may be NULL: all 0) of every model m under one key `seed`, in
 * ONE persistent launch: the models are queued heaviest first (descending
 * packets[m], ties by index), and each CTA takes the first queued model
 * that still has packet ids, stages that model's tables, runs its warps on
 * it until its ids run out, and moves on, so the models' tails overlap and
 * the longest packets start early. CTAs are at most 256 threads
 * (tune->block; KRL_ERR_ARG above). Each packet's
 * random stream, and therefore every tally, is exactly what krl_run_packets
 * on that grid with the same (seed, ids) gives. Tallies accumulate into each
 * grid. records (host [n_models] of device pointers, or NULL; a NULL entry
 * skips that model): model m's packet records, records[m][id - first_ids[m]],
 * as krl_run_packets writes them. stats (host [n_models] or NULL): per-model
 * counters; when given the call synchronises `s`. The call first waits for `s` (it rewrites a pinned
 * argument mirror the previous run's copy reads), then enqueues a copy of
 * the arguments, the launch and the counter updates; captured into a CUDA
 * graph (stats must then be NULL, and the stream must be idle when the
 * capture begins), each replay copies the arguments of the captured call
 * again and reruns the same packets.
 */
KRL_API krl_status krl_batch_run(krl_batch* b, const uint64_t* packets, const uint64_t* first_ids, uint64_t seed,
                                 const krl_tune* tune, krl_packet_record* const* records, krl_run_stats* stats,
                                 krl_stream s);

/* ------------------------------------------------------------------ channel maps */

typedef struct {
    int camera;             /* >= 0: the line's camera `camera` (direction from
                               cam_theta/cam_phi; emissivity defaults to this
                               grid's tally for it); -1: use theta/phi below    */
    double theta, phi;      /* camera direction when camera == -1              */
    int npix_x, npix_y;     /* pixels, >= 1                                     */
    double fov_cells;       /* image width in cell units (square pixels)       */
    const float* emiss;     /* device [ncell][n_ch] camera-directed scattering
                               emissivity (raw KRL_OUT_EMISS units), or NULL for
                               this grid's tally of `camera`; 4-byte aligned.
                               When 16-byte aligned and n_ch is 4, 8, 16, 32,
                               64 or 128, each cell's row is read as 16-byte
                               vectors (faster; the same result)              */
    const float* jline;     /* device [ncell] frequency-integrated line emission
                               per unit path (same units), or NULL              */
    int no_scratch;         /* nonzero: allocate nothing; evaluate the profile
                               per segment (slower, same result)                */
} krl_raytrace_desc;

/*
 * Deterministic ray trace of channel maps (Sec. 2.2.2, Eq. imaging-formal,
 * Eq. imaging-alphas): orthographic, pixel-centred parallel rays along the
 * camera direction n, image axes (e_theta, e_phi), centred on the box, no
 * incoming intensity; per cell segment dl and channel k (the line's
 * v_k = v_min + (k + 1/2) dv, 1 <= n_ch <= 128) with x_k = -(v_k + n.V)/b:
 * I <- I e^{-dtau} + j_k dl (1 - e^{-dtau})/dtau, dtau = (alpha0 H(a, x_k) +
 * tau_abs) dl (tau_abs: the grid's continuum, zero without one),
 * j_k = emiss_k + jline H(a, x_k)/sqrt(pi). maps: device float32
 * [n_ch][npix_y][npix_x], written (raw units: emissivity x cell widths).
 * All faces are open for the rays. Enqueued on `s`; does not synchronise.
 * alpha_k depends on the cell and the channel only, so it is tabulated once
 * per call in a stream-ordered scratch of ncell x n_ch floats, beside each
 * ray's starting cell and position (32 bytes per pixel, set up in FP64 once
 * per ray) (cudaMallocAsync on `s`, freed on `s` after the trace); with
 * no_scratch, or when that memory is not available, the trace evaluates H per
 * segment and each ray's lanes set it up themselves, with the same result.
 */
KRL_API krl_status krl_raytrace_channels(krl_grid* g, const krl_raytrace_desc* d, float* maps, krl_stream s);

/* ------------------------------------------------------------------ no allocation */

/*
 * Volume-source emission CDF without any device allocation. The paper has
 * no counterpart: this is a service to callers that cannot call cudaMalloc,
 * such as a host application that hands all device memory to its own pool
 * or framework allocator (a raw cudaMalloc there may fail or fragment the
 * pool), or a latency-critical loop that must not take cudaMalloc's
 * implicit device synchronisation.
 *
 * Computes cdf[i] = (rate[0] + ... + rate[i]) / (rate[0] + ... + rate[n-1])
 * in FP64 -- the same table krl_line_set builds for KRL_SRC_VOLUME and
 * krl_tallies_get(KRL_OUT_SRC_CDF) returns. rate: device float32 [n],
 * borrowed; cdf: device double [n], written. 1 <= n <= 2^27 cells; larger n
 * is rejected with KRL_ERR_ARG.
 *
 * The scan's scratch (65537 partial sums and a flag, about 512 KiB) is a
 * fixed array in the library's device image: every GPU that loads the
 * library holds it until the process exits, and the call allocates nothing
 * (no cudaMalloc, no cudaFree). The first call on a device looks up that
 * array's device address once (cudaGetSymbolAddress); make that first call
 * before any stream capture. All calls share the array and it keeps the
 * last call's contents (the call clears what must start at zero), so calls
 * that overlap on the GPU -- on different streams or threads -- race and
 * must be serialised by the caller.
 *
 * Synchronises `s` to report bad input: KRL_ERR_NUMERIC for a NaN, Inf or
 * negative rate, KRL_ERR_ARG for a zero total or NULL pointers.
 */
KRL_API krl_status krl_emission_cdf_noalloc(const float* rate, int n, double* cdf, krl_stream s);

#ifdef __cplusplus
}
#endif

#endif /* KRL_H */
