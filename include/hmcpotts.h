/*
 * hmcpotts.h -- C ABI of the GB300 (sm_103a) hybrid Monte Carlo grain-growth
 * library: checkerboard Potts sweep driven by a stored-energy field from
 * Monte Carlo crystal plasticity (Zhang, Dingreville, Bartel, Lusk,
 * "Hybrid Monte Carlo Simulation of Stress-Induced Texture Evolution with
 * Inelastic Effects", arXiv 1007.3509).
 *
 * Conventions
 *  - Every call returns int: HP_OK (0) or a negative HP_ERR_* code.  A failed
 *    call leaves a message readable with hp_last_error_message().
 *  - Pointers documented "device" are CUDA device pointers; "host" pointers
 *    are ordinary host memory.  Device buffers passed to hp_bind() and
 *    hp_set_field() are BORROWED: the caller owns them and keeps them alive
 *    until hp_destroy() or until they are re-bound.  Everything else the
 *    library allocates itself and frees in hp_destroy().
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  GPU calls are asynchronous on that stream unless documented
 *    otherwise.  A handle may be used from one host thread at a time.
 *  - Lattices are periodic boxes with even edges, linear site index
 *    x + Lx*(y + Ly*z), int32 grain ids q (the Potts spins of Eq. (7)).
 *  - Energies inside the sweep are int32 fixed point: 256 units = 1 J, the
 *    interaction energy unit of Eq. (7).
 */
#ifndef HMCPOTTS_H
#define HMCPOTTS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HP_API __attribute__((visibility("default")))
#else
#define HP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define HP_OK 0
#define HP_ERR_ARG (-1)      /* invalid argument or unsupported combination      */
#define HP_ERR_CUDA (-2)     /* a CUDA runtime call or kernel launch failed      */
#define HP_ERR_OOM (-3)      /* device allocation failed                         */
#define HP_ERR_TIMEOUT (-4)  /* a bounded device-side wait gave up               */
#define HP_ERR_STATE (-5)    /* call made in the wrong order (e.g. nothing bound) */
#define HP_ERR_CHECKSUM (-6) /* checkpoint file corrupted                        */

/* Field modes: where the per-site bulk energy b_i of Eq. (7) comes from.     */
#define HP_FIELD_NONE 0   /* b = 0                                             */
#define HP_FIELD_GRAIN 1  /* b_i = table[q_i]  (one energy per grain, G entries) */
#define HP_FIELD_POINT 2  /* b_i = table[mp_i] (one energy per material point;   */
                          /*  mp is carried with q when a boundary sweeps a site) */

/* Orientation kinds. */
#define HP_ORIENT_ANGLE 0 /* one rotation angle about z in [0, pi/2), float[G]  */
#define HP_ORIENT_SO3 1   /* unit quaternion (w,x,y,z) uniform on SO(3), float[4G] */
#define HP_ORIENT_ZROT 2  /* quaternion (cos t/2, 0, 0, sin t/2) of a rotation by the */
                          /* HP_ORIENT_ANGLE angle t about z (Sec. 5), float[4G]     */

/* Sweep kernel choice (hp_set_sweep_kernel). */
#define HP_SWEEP_AUTO 0   /* fused multi-phase tiles where available            */
#define HP_SWEEP_PHASE 1  /* one launch per colour phase, in place              */
#define HP_SWEEP_FUSED 2  /* all phases of a plane in shared memory, double-buffered */

typedef struct {
    int32_t dim;        /* 2 or 3                                             */
    int64_t L[3];       /* edges; even; L[2] ignored (treated as 1) in 2D     */
    int32_t nbr;        /* neighbours M: 4 or 8 in 2D, 6 or 26 in 3D          */
    int32_t J_fix;      /* interaction energy J in fixed point (J = 1 -> 256) */
    uint64_t seed;      /* Philox4x32-10 key of this lattice                  */
    int32_t n_grains;   /* G: grain ids are 0..G-1                            */
    int32_t field_mode; /* HP_FIELD_*                                         */
} hp_desc;

typedef struct hp_handle hp_handle;

/* Latest error message of this thread (never NULL). */
HP_API const char* hp_last_error_message(void);

/* Copy this thread's latest error message into buf (capacity n bytes, always
 * NUL-terminated, truncated if longer).  Messages are kept per host thread, so
 * h may be NULL.  HP_ERR_ARG (without touching the message) if buf is NULL or
 * n is 0.                                                                    */
HP_API int hp_last_error(const hp_handle* h, char* buf, size_t n);

/* Library build/version string (never NULL). */
HP_API const char* hp_version(void);

/* Number of CUDA kernel launches this library has issued in this process
 * (all threads, all handles); for accounting in benchmarks.                  */
HP_API int hp_kernel_launches(uint64_t* out);

/* Create a lattice handle.  Validates the descriptor (Sec. 4: square or cubic
 * lattice, M neighbours; colour count follows from nbr: 2 for 4/6, 4 for 2D-8,
 * 8 for 3D-26).  No device memory is touched.                                */
HP_API int hp_create(const hp_desc* desc, hp_handle** out);

/* Free everything the library allocated for the handle.  Safe with NULL.      */
HP_API int hp_destroy(hp_handle* h);

/* Bind the caller's device buffers: q (int32[N], required) and mp (int32[N],
 * required in HP_FIELD_POINT mode, else may be NULL).  Allocates the library's
 * double-buffer copies (same sizes) used by the fused sweep.                  */
HP_API int hp_bind(hp_handle* h, int32_t* q, int32_t* mp);

/* Lattice state in and out (Sec. 4: the Potts spins q_i and, Sec. 6, the
 * material point each site carries).  hp_set_spins copies N ids into the bound
 * q (and N material-point indices into the bound mp when mp is not NULL) from
 * host memory (is_host != 0; pinned memory makes the copy asynchronous) or
 * from device memory; hp_get_spins copies them out the same way.  Ids are not
 * checked here: a lattice holding ids outside 0..G-1 is reported by
 * hp_grain_counts / hp_measure, and the sweep clamps every table index.
 * HP_ERR_STATE if nothing is bound (or mp is given but no mp buffer is bound).
 * Asynchronous on `stream`: host buffers must stay valid until it completes. */
HP_API int hp_set_spins(hp_handle* h, const int32_t* q, const int32_t* mp, int32_t is_host, void* stream);
HP_API int hp_get_spins(const hp_handle* h, int32_t* q, int32_t* mp, int32_t is_host, void* stream);

/* Initial polycrystal (Sec. 4-5 set-up): Voronoi tessellation of G seeds.
 * Seeds are drawn in rounds from Philox(seed; g, round, tag 2 | 0); a site
 * drawn by several seeds goes to the lowest g, losers redraw.  Every site gets
 * the seed at the smallest periodic minimum-image squared integer distance,
 * ties to the lowest index.  Writes q, sets mp to the identity when bound, and
 * writes G orientations of `orient_kind` into orient (device float[G] or
 * float[4G]; may be NULL) and the seed sites into seed_pos (device int64[G];
 * may be NULL).  Synchronises `stream` once per seeding round.               */
HP_API int hp_init_voronoi(hp_handle* h, int32_t orient_kind, float* orient, int64_t* seed_pos, void* stream);

/* Same tessellation as hp_init_voronoi (bit-identical q, seed_pos, orient),
 * but it allocates no device memory: no cudaMalloc, cudaFree or allocating
 * library routine is called.  The paper has no counterpart; this entry point
 * exists for callers that cannot allocate while they run, such as a process
 * whose device memory is all pre-reserved by another allocator, or a
 * steady-state loop that must never enter the allocator.
 * Scratch (seed coordinates, cell lists and counters) lives in one file-scope
 * device array of HP_VORONOI_STATIC_BYTES (16 MiB) that every GPU loading the
 * library holds until exit; G above HP_VORONOI_STATIC_MAX_GRAINS is rejected
 * with HP_ERR_ARG.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device.  The call reads a counter back
 * to the host and synchronises `stream` once per seeding round, so it must
 * never be made while the stream is being captured into a CUDA graph.  All
 * calls share the one array and each call clears what it needs, so calls that
 * overlap on the GPU (concurrent streams, several host threads) race and must
 * be serialised by the caller.                                               */
#define HP_VORONOI_STATIC_BYTES (16u << 20)
#define HP_VORONOI_STATIC_MAX_GRAINS 262144
HP_API int hp_init_voronoi_static(hp_handle* h, int32_t orient_kind, float* orient, int64_t* seed_pos, void* stream);

/* Orientations only (same draws as hp_init_voronoi).                          */
HP_API int hp_orientations(int32_t G, uint64_t seed, int32_t orient_kind, float* orient, void* stream);

/* Stored-energy field table (borrowed device int32): G entries in
 * HP_FIELD_GRAIN mode, N entries (one per material point) in HP_FIELD_POINT.
 * HP_ERR_STATE for a HP_FIELD_NONE handle; HP_ERR_ARG when n is not G or N.
 * Host-only bookkeeping: the table is read by the next sweep.                */
HP_API int hp_set_field(hp_handle* h, const int32_t* table, int64_t n);

/* Misorientation-dependent interaction energy and mobility (the pair energy
 * J_{q_i,q_n} of Eq. (7); the arbitrary-misorientation extension the paper
 * names in Sec. 6).  angle: device int32[G] (borrowed), each grain's
 * orientation as an integer angle in [0, period) (e.g. millidegrees of a
 * rotation about z, period 90000 for a cubic crystal).  The misorientation of
 * grains a and b is min(d, period - d), d = |angle_a - angle_b|; its bin is
 * misorientation / bin, clamped to nbins - 1 (the bins must cover [0,
 * period/2]).  J: host int32[nbins] energies per bin in [0, 2^20] (256 = 1 J);
 * mobility: host uint32[nbins] relative mobilities (0xFFFFFFFF = 1) or NULL.
 * A site's energy in state s is the sum over neighbours n with q_n != s of
 * J[bin(s, q_n)]; d = E(q_j) - E(q_i) + (b_j - b_i); the threshold of the
 * trial is scaled by the mobility m of the (q_i, q_j) boundary: eff = thr[d]
 * (0xFFFFFFFF for d < 0) if m is 0xFFFFFFFF, m if thr[d] is, else
 * floor(thr[d] m / 2^32); accept iff d <= D and (eff == 0xFFFFFFFF or u1 < eff).
 * With tables set, hp_sweep runs the per-colour kernel; angle = J = NULL
 * clears them (back to the constant J_fix).  Copies the tables; synchronises
 * `stream`.                                                                  */
HP_API int hp_set_anisotropy(hp_handle* h, const int32_t* angle, int32_t period, int32_t bin, int32_t nbins,
                             const int32_t* J, const uint32_t* mobility, void* stream);

/* Grain angles in the integer units of hp_set_anisotropy: out[g] =
 * floor(theta_g [degrees] * unit_per_degree) mod period, theta_g the angle of
 * HP_ORIENT_ANGLE (device float[G]) or the rotation angle 2 atan2(z, w) of
 * HP_ORIENT_ZROT (device float[4G]); out device int32[G].                    */
HP_API int hp_angle_units(int32_t G, int32_t orient_kind, const float* orient, int32_t unit_per_degree,
                          int32_t period, int32_t* out, void* stream);

/* Read-Shockley tables, host FP64: bin k has the misorientation
 * theta = (k + 1/2) bin / unit_per_degree degrees, x = theta / theta_max;
 * J_out[k] = round-half-even(256 J_max x (1 - ln x)) for x < 1, 256 J_max
 * beyond; mob_out (may be NULL) = floor(2^32 (1 - exp(-5 x^4))), saturated at
 * 0xFFFFFFFF (low-angle boundaries slow).                                    */
HP_API int hp_build_read_shockley(double J_max, double theta_max, int32_t bin, int32_t nbins, int32_t unit_per_degree,
                                  int32_t* J_out, uint32_t* mob_out);

/* Parametric links between the sharp-interface and Monte Carlo models, Eq. (8)
 * (Sec. 3): from the physical boundary stiffness gamma_s [J/m^2] and mobility
 * m_s [m^4/(J s)], the length of one lattice unit l0 [m], and the Monte Carlo
 * counterparts gamma_mc (stiffness in units of J per lattice spacing) and m_mc
 * (mobility in lattice units per MCS) at the run's temperature, with lattice
 * spacing Delta, interaction energy J and time step tau_mc (1 MCS = tau_mc):
 *   E0 = gamma_s Delta^2 J l0^2 / gamma_mc
 *   t0 = Delta^4 m_mc l0^4 / (J tau_mc E0 m_s),  seconds per MCS = tau_mc t0
 *   b (MC units) = b_per_bs * b_s  with  b_per_bs = Delta^3 l0^3 / (2 E0)
 * so a physical bulk energy density b_s [J/m^3] becomes the field of Eq. (7)
 * and each MCS a physical time (the paper's Sec. 5 runs take 1 MCS = 10 min). */
typedef struct {
    double gamma_s, m_s, l0;     /* physical stiffness, mobility, lattice unit   */
    double gamma_mc, m_mc;       /* Monte Carlo stiffness and mobility           */
    double Delta, J, tau_mc;     /* lattice spacing, interaction energy, MC step */
} hp_si_in;
typedef struct {
    double E0, t0;               /* characteristic energy [J] and time [s]       */
    double seconds_per_mcs;      /* physical time of one MCS                     */
    double b_per_bs;             /* MC bulk energy per unit physical b_s [J/m^3] */
} hp_si_out;
HP_API int hp_si_links(const hp_si_in* in, hp_si_out* out);

/* Metropolis threshold table, host FP64 (Sec. 4, acceptance
 * min(1, exp(-dE/kT))): out[0] = 0xFFFFFFFF (dE = 0 accepted) or 0 when
 * zero_rule = 1; out[d] = min(floor(2^32 exp(-d/(256 kT))), 0xFFFFFFFE) for
 * d >= 1 up to *D, the last nonzero entry (D = 0 when kT = 0).  `cap` is the
 * capacity of out; HP_ERR_ARG if the table does not fit.                     */
HP_API int hp_build_threshold_table(double kT, int32_t zero_rule, uint32_t* out, int32_t cap, int32_t* D);

/* Copy a threshold table (host uint32[D+1]) to the device for this handle.   */
HP_API int hp_set_threshold_table(hp_handle* h, const uint32_t* thr, int32_t D, void* stream);

/* Choose the sweep kernel (HP_SWEEP_*); both give bit-identical lattices.    */
HP_API int hp_set_sweep_kernel(hp_handle* h, int32_t kind);

/* Run n_mcs Monte Carlo steps (Sec. 4): each step runs colours 0..C-1 in
 * order; a colour phase updates all its sites from the state left by the
 * previous phase.  Site i of colour c draws Philox(seed; i, sweep, tag 0 | c),
 * proposes neighbour k = (u0*M)>>32, and with q_j != q_i computes
 * d = J_fix*(#nbrs equal q_i - #nbrs equal q_j) + (b_j - b_i); accepts if
 * d < 0, rejects if d > D, else accepts iff thr[d] = 0xFFFFFFFF or u1 < thr[d].
 * An accepted site copies q_j and mp_j (Sec. 6: the swept site takes the
 * content of the overtaking grain).  `sweep` starts at the handle's counter,
 * which advances by n_mcs.  On return the state is in the bound buffers.     */
HP_API int hp_sweep(hp_handle* h, int32_t n_mcs, void* stream);

/* Tile variants of the fused sweep kernel, all giving identical lattices:
 * plane tiles (parity-split window, variants 0-2 in 2D, 0-3 in 3D), lean tiles
 * (row-major windows fed by bulk copies, 3-5 in 2D, 4-7 in 3D) and, for the
 * 26-neighbour lattice, lean 3D windows (64 x 44, 40, 36, 32: variants 8-11;
 * every random number drawn while the window is in flight).  Until a variant is
 * chosen, a handle sweeps with the fastest measured for its kind of lattice:
 * variant 11 in 3D with material points, 8 in 3D without, 4 in 2D.
 * hp_sweep_variants: how many exist for `nbr`.
 * hp_set_sweep_variant: choose one (HP_ERR_ARG if not built for the handle's
 * field mode).  hp_sweep_autotune: time every variant for n_mcs MCS on a
 * backup of the bound state (the lattice and sweep counter are restored),
 * keep the fastest, write per-variant milliseconds to ms_out (host float[n],
 * -1 for unavailable variants; may be NULL) and the choice to *chosen.
 * Allocates a temporary copy of the lattice; synchronises `stream`.          */
HP_API int hp_sweep_variants(int32_t nbr, int32_t* n);
HP_API int hp_set_sweep_variant(hp_handle* h, int32_t v);
HP_API int hp_sweep_autotune(hp_handle* h, int32_t n_mcs, float* ms_out, int32_t* chosen, void* stream);
/* Synchronous: HP_ERR_TIMEOUT if a TMA-fed sweep kernel since the last call
 * gave up waiting for one of its window copies (every such wait is bounded, about
 * two seconds); clears the flag.  *timed_out = 1: the block then waited up to
 * four more limits for the copies in flight and they landed before it left (the
 * lattice written by that launch is wrong, the context is sound); 2: even that
 * drain ran out, copies may have landed after the block left and the CUDA
 * context should not be trusted further.  0 and HP_OK otherwise.             */
HP_API int hp_sweep_status(int32_t* timed_out);

/* Test hook of the timeout paths, no counterpart in the paper: one block waits
 * on an mbarrier with nothing in flight (no copy or tensor-core operation) and
 * a limit of limit_cycles (1 .. 2^32 SM clocks).  The one arrival it expects
 * comes after two limits when late != 0 (the first wait gives up, the drain
 * sees the arrival: flag 1) or never (the drain runs out too: flag 2).  The
 * flag is raised exactly as by a sweep (unit 0, read by hp_sweep_status) or
 * surrogate (unit 1, hp_mlp_status) kernel that timed out; since nothing was in
 * flight, the context stays sound either way.  Asynchronous on `stream`.     */
HP_API int hp_debug_wait_timeout(int32_t unit, int64_t limit_cycles, int32_t late, void* stream);

/* The handle's MCS counter: the `sweep` word of the draws of the next MCS
 * (Philox counter word 2).  Setting it replays or continues a run from any
 * step; it takes effect at the next hp_sweep.  Host only; HP_ERR_ARG on NULL. */
HP_API int hp_get_sweep_counter(const hp_handle* h, uint64_t* out);
HP_API int hp_set_sweep_counter(hp_handle* h, uint64_t value);

/* Per-grain site counts (device int64[G]) and the number of grains with a
 * nonzero count (device int32[1]) of the bound lattice (Sec. 4: average grain
 * size N / alive).                                                           */
HP_API int hp_grain_counts(hp_handle* h, int64_t* counts, int32_t* alive, void* stream);

/* Texture (Sec. 5): per-grain bins of the orientations and the area-weighted
 * histogram hist[b] = sum of counts of grains in bin b (device int64).
 * HP_ORIENT_ANGLE: 90 one-degree bins of the angle; bins int32[G].
 * HP_ORIENT_SO3: 20 bins of the max Schmid factor over [0, 0.5] followed by
 * 4 bins (none, <100>, <110>, <111> within 15 degrees of the loading axis x);
 * bins int32[2G]; hist int64[24].  HP_ORIENT_ZROT: 90 one-degree bins of the
 * rotation angle 2 atan2(z, w); bins int32[G]; hist int64[90].               */
HP_API int hp_texture(int32_t G, int32_t orient_kind, const float* orient, const int64_t* counts, int32_t* bins,
               int64_t* hist, void* stream);

/* One synchronous measurement of a bound lattice (Sec. 4 average grain size
 * N / (grains alive); Sec. 5 texture and the bulk energy the grains carry).
 * With accumulate = 0 the stats (and hist) are reset first; with accumulate
 * != 0 this lattice's sums are added to them, so one struct can gather an
 * ensemble of lattices.  Integer sums are exact; the derived doubles are
 * recomputed from the accumulated sums on every call.                        */
typedef struct {
    int64_t sites;      /* sites measured                                       */
    int64_t alive;      /* grains with at least one site (summed over lattices) */
    double mean_area;   /* sites / alive: average grain size in sites            */
    int64_t field_sum;  /* sum over sites of the field b_i (fixed point, 256 = 1 J):
                           table[q_i] (HP_FIELD_GRAIN), table[mp_i] (HP_FIELD_POINT),
                           0 (HP_FIELD_NONE)                                      */
    double mean_field;  /* field_sum / 256 / sites: volume-weighted bulk energy [J] */
    int64_t hist_total; /* sites in the texture histogram (its first block)       */
    double families[4]; /* HP_ORIENT_SO3: volume fractions with no family, <100>,
                           <110>, <111> within 15 degrees of the loading axis x   */
    double mean_mmax;   /* HP_ORIENT_SO3: volume-weighted mean max Schmid factor
                           from the 20 bin centres                                */
} hp_stats;
/* orient (device, as for hp_texture; NULL skips the texture): the histogram of
 * hp_texture (24 bins for HP_ORIENT_SO3, 90 otherwise) is added into hist
 * (host int64[n_bins], may be NULL).  Device scratch for the counts, bins and
 * histogram is allocated on the first call and kept by the handle.  Returns
 * HP_ERR_STATE if the lattice holds ids outside 0..G-1 (stats untouched), if
 * nothing is bound, or if the handle's field table is not set.              */
HP_API int hp_measure(hp_handle* h, int32_t orient_kind, const float* orient, int32_t accumulate, hp_stats* stats,
                      int64_t* hist, int32_t n_bins, void* stream);

/* Orientation-dependent Gaussian bulk energy of Eq. (9) (Sec. 5, Fig. 3): a
 * grain with angle t (device float[G], HP_ORIENT_ANGLE) has orientation
 * n = floor(t in degrees) + 1 and b = round-half-even(256 scale e(n)) with
 * e(n) = (32 pi)^(-1/2) exp(-(n - 46)^2 / (2 46^2)) [J]; b_out device int32[G]. */
HP_API int hp_gaussian_field(int32_t G, const float* angle, double scale, int32_t* b_out, void* stream);

/* Texture fit of Eq. (10), host FP64: the 90 one-degree angle bins, folded so
 * that angles above 45 degrees count as negative (Sec. 5), normalised to a
 * density per degree, and fitted by least squares to
 * f(phi) = exp(-phi^2 / (2 g^2)) / (g sqrt(2 pi)); returns g [degrees] and the
 * residual sum of squares (may be NULL).                                     */
HP_API int hp_texture_fit(const int64_t* hist, int32_t n_bins, double* g_out, double* residual_out);

/* Checkpoint / resume of a handle's lattice state: q (and mp when bound), the
 * sweep counter and the descriptor, followed by a CRC-32.  Field and threshold
 * tables are caller inputs and are not stored.  Loading into a handle with a
 * different descriptor fails with HP_ERR_ARG; a corrupted or truncated file
 * with HP_ERR_CHECKSUM.  Both synchronise `stream`.  Because every draw is
 * keyed by (seed, sweep, colour, site), resuming is bit-exact.               */
HP_API int hp_checkpoint_save(hp_handle* h, const char* path, void* stream);
HP_API int hp_checkpoint_load(hp_handle* h, const char* path, void* stream);

/* Closed-form per-grain field under uniaxial stress sigma [MPa] along x
 * (Sec. 5): d = loading axis in the crystal frame, E(d) the directional
 * Young's modulus of cubic (C11, C12, C44) [MPa], w = sigma^2/(2 E(d)),
 * m_max = largest FCC {111}<110> Schmid factor of d; the energy
 * e = energy_scale * (w + k_disl * m_max) [J] is quantised to
 * b = round-half-even(256 e) clamped to +-2^20.  quat: device float[4G];
 * b_out device int32[G]; w_out, mmax_out device float[G] or NULL.           */
HP_API int hp_grain_field(int32_t G, const float* quat, double C11, double C12, double C44, double sigma,
                   double k_disl, double energy_scale, int32_t* b_out, float* w_out, float* mmax_out,
                   void* stream);

/* Philox4x32-10 of n counters (device uint32[4n]) into out (device uint32[4n]),
 * the generator every kernel here draws from (exposed for verification).     */
HP_API int hp_philox(uint64_t seed, const uint32_t* ctr, int64_t n, uint32_t* out, void* stream);

/* ------------------------------------------------------------------------ */
/* Ensembles: many independent lattices of uneven size, temperature, load and  */
/* seed swept together (the paper averages 10-100 independent runs, Sec. 4-5). */
/* ------------------------------------------------------------------------ */
typedef struct hp_ensemble hp_ensemble;

/* Group R handles (borrowed; each already bound, with its threshold table and
 * field set) that share dim, nbr, field mode and whether mp is bound.  Every
 * member keeps its own seed, sweep counter, temperature (threshold table) and
 * field.                                                                       */
HP_API int hp_ensemble_create(hp_handle* const* members, int32_t R, hp_ensemble** out);
/* Free the ensemble's graph, capture stream and device argument arrays; the
 * members stay valid and belong to the caller.  Safe with NULL.              */
HP_API int hp_ensemble_destroy(hp_ensemble* e);
/* Tile variant used by hp_ensemble_sweep (default 0); HP_ERR_ARG for a variant
 * not built for the members' field mode.  Lean 3D windows of an ensemble are
 * filled by 16-byte asynchronous copies (no tiled TMA descriptors per member). */
HP_API int hp_ensemble_set_variant(hp_ensemble* e, int32_t v);
/* Pick the fastest tile variant for the whole ensemble (state restored).      */
HP_API int hp_ensemble_autotune(hp_ensemble* e, int32_t n_mcs, float* ms_out, int32_t* chosen, void* stream);
/* Sweep every member n_mcs MCS, bit-identical to hp_sweep on each member.  All
 * replicas share each launch (one CTA per replica tile); the n_mcs launches are
 * captured once into a CUDA graph (re-captured when n_mcs or the variant
 * changes) and replayed as one graph launch on `stream`.                      */
HP_API int hp_ensemble_sweep(hp_ensemble* e, int32_t n_mcs, void* stream);

/* ------------------------------------------------------------------------ */
/* Monte Carlo crystal plasticity (Sec. 2, Eqs. (1)-(3), Table 1) and the     */
/* per-point field of Eq. (4).                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    double C11, C12, C44;    /* cubic moduli [MPa]                              */
    double tau0, taus, h0;   /* Voce hardening: g = taus - (taus-tau0) exp(-h0 gamma/(taus-tau0)) */
    double beta;             /* inverse temperature of Eq. (1) [per MJ/m^3]     */
    double G;                /* shear modulus of Eq. (4) [MPa]                  */
    double e_incr;           /* strain increment e of Eq. (3)                   */
    double energy_scale;     /* J (MC units) per MJ/m^3 for the field           */
    double w_weight;         /* weight of the elastic energy in the field: 1 for */
                             /* w + E_rho, 0 for the plastic driving force alone */
                             /* (Sec. 5 suppresses the elastic one)              */
} hp_cp_params;

/* Material-point state, structure of arrays over P points (device memory):
 * eps_p float[6][P] (components xx yy zz yz xz xy, crystal frame), gamma
 * float[P] (accumulated slip), g float[P] (slip resistance).                 */
typedef struct {
    int64_t P;
    float* eps_p;
    float* gamma;
    float* g;
} hp_cp_state;

/* The single-slip return map as the plasticity kernels evaluate it, for
 * testing: x[i] (device double[n]) = the slip of a system with resolved shear
 * at[i] > g[i] (device float[n] each) and k[i] = P:C:P (device double[n]), the
 * root of at - k x = g(gamma + x) for the Voce law of prm (tau0, taus, h0),
 * x = (at - g)/k without hardening.                                          */
HP_API int hp_debug_return_map(const hp_cp_params* prm, const float* at, const float* g, const double* k, int64_t n,
                               double* x, void* stream);

/* Zero plastic strain and slip, g = tau0.                                    */
HP_API int hp_cp_reset(const hp_cp_params* prm, hp_cp_state* st, void* stream);

/* Apply load increments t = t0+1 .. t0+n_incr to every point (Eq. (3), Taylor:
 * total strain t e diag(1,-1/2,-1/2) in the sample frame).  Point p has the
 * orientation quat[4*grain[p]].  Per increment: trial stress, candidate set
 * |tau_alpha| > g, single-slip return map per candidate (FP64 Newton), energies
 * E_alpha, Boltzmann probabilities (Eq. (1)) and the pick of Eq. (2) with
 * R = u0/2^32 of Philox(seed; p, t, tag 1).  Afterwards, optionally writes
 * sigma (device float[6][P], NULL to skip), w and E_rho (device float[P] each,
 * NULL to skip; E_rho = 2 g^2/G, w = 1/2 sigma : C^-1 : sigma) and the
 * quantised field b = round-half-even(256 energy_scale (w_weight w + E_rho)) (device
 * int32[P], NULL to skip) for HP_FIELD_POINT.                                */
HP_API int hp_cp_step(const hp_cp_params* prm, uint64_t seed, const int32_t* grain, const float* quat, uint32_t t0,
               int32_t n_incr, hp_cp_state* st, float* sigma, float* w, float* erho, int32_t* b, void* stream);

/* Periodic elastic equilibrium of the polycrystal (Sec. 5: the plasticity is
 * coupled to a deformation solver and every load increment is iterated to
 * quasi-static equilibrium).  One material point per voxel of an n[0] x n[1] x
 * n[2] grid (linear index x + n0 (y + n1 z), edges powers of two up to 1024).
 * Solves sigma = C(x) : (eps - eps_p), div sigma = 0, <eps> = E by the
 * Moulinec-Suquet fixed point with the isotropic reference medium mu0 = (C44 +
 * (C11 - C12)/2)/2, lambda0 = (C11 + 2 C12)/3 - 2 mu0/3; the strain fluctuation
 * is zero on the Nyquist planes.  C(x): cubic (prm C11, C12, C44) rotated by
 * quat[4 grain[x]]; eps_p: crystal-frame plastic strain, device float[6][N]
 * (the hp_cp_state layout; NULL = none); E: host double[6] sample-frame mean
 * strain; eps: device float[6][N] sample-frame strain, the initial guess on
 * entry (or set to E first when start_from_mean) and the solution on return;
 * sigma (device float[6][N], may be NULL): the sample-frame stress.  Stops
 * when the largest change of a strain component in one iteration is below
 * tol max|E| or after max_iter; *iters and *change (may be NULL) report the
 * iteration count and the last relative change.  FP32; allocates its work
 * buffer (six complex fields, 48 bytes per voxel) for the call; synchronous.
 * Voigt order xx yy zz yz xz xy, tensor components throughout.              */
typedef struct {
    int32_t n[3];
    double tol;
    int32_t max_iter;
    int32_t start_from_mean;
} hp_elastic_params;
HP_API int hp_elastic_solve(const hp_cp_params* prm, const hp_elastic_params* ep, const int32_t* grain,
                            const float* quat, const float* eps_p, const double E[6], float* eps, float* sigma,
                            int32_t* iters, double* change, void* stream);

/* One load increment t of every material point with the point's own total
 * strain (sample frame, device float[6][P], e.g. from hp_elastic_solve) in
 * place of the Taylor strain of hp_cp_step; otherwise as hp_cp_step with
 * n_incr = 1 (the draws are keyed by t).                                     */
HP_API int hp_cp_step_strain(const hp_cp_params* prm, uint64_t seed, const int32_t* grain, const float* quat,
                             uint32_t t, const float* eps_total, hp_cp_state* st, float* sigma, float* w, float* erho,
                             int32_t* b, void* stream);

/* Deterministic rate-independent multi-slip crystal plasticity: the model the
 * Monte Carlo plasticity is checked against (Sec. 2, Fig. 1, a nickel single
 * crystal; the ill-conditioned constraint equations of the active systems are
 * solved with a singular value decomposition).  FP64, one thread per point.
 * Per increment (crystal frame, prm C11 C12 C44 tau0 taus h0, Voce hardening
 * g(gamma) as for hp_cp_step; beta, G, energy_scale and w_weight unused):
 * trial stress C : (eps - eps_p), active set {a : |tau_a| - g(gamma) > tol},
 * tol = 1e-12 tau0; Newton on |tau_a| - sum_b s_a s_b P_a:C:P_b x_b =
 * g(gamma + sum x) with the Moore-Penrose inverse of the constraint matrix
 * (eigenvalues at or below 1e-10 of the largest discarded); drop systems whose
 * slip comes out negative, add systems whose resolved shear then exceeds g,
 * repeat; commit eps_p += sum x_a s_a P_a, gamma += sum x_a.
 * State, device memory: eps_p double[6][P] (xx yy zz yz xz xy, crystal frame),
 * gamma double[P].                                                           */
typedef struct {
    int64_t P;
    double* eps_p;
    double* gamma;
} hp_det_state;

/* Zero plastic strain and accumulated slip.                                  */
HP_API int hp_det_reset(hp_det_state* st, void* stream);

/* Load increments t = t0+1 .. t0+n_incr of the prescribed strain
 * t e_incr diag(1,-1/2,-1/2) (sample frame, as hp_cp_step); point p has the
 * orientation quat[4*grain[p]].  Afterwards sigma (device double[6][P],
 * crystal frame; NULL to skip) holds the stress and n_active (device int32[P],
 * NULL to skip) the number of active systems of the last increment, or -1 when
 * the active set did not settle within 50 passes: that point's state is then
 * left as before the failing increment and its later increments are skipped.
 * Asynchronous on stream.                                                    */
HP_API int hp_det_step(const hp_cp_params* prm, const int32_t* grain, const float* quat, uint32_t t0,
                       int32_t n_incr, hp_det_state* st, double* sigma, int32_t* n_active, void* stream);

/* One increment to each point's own total strain (sample frame, device
 * float[6][P], e.g. from hp_elastic_solve); otherwise as hp_det_step.       */
HP_API int hp_det_step_strain(const hp_cp_params* prm, const int32_t* grain, const float* quat,
                              const float* eps_total, hp_det_state* st, double* sigma, int32_t* n_active,
                              void* stream);

/* ------------------------------------------------------------------------ */
/* Learned field surrogate: 11 -> 64 -> 64 -> 64 -> 2 perceptron with GELU,    */
/* BF16 operands and FP32 accumulation on the tensor cores.  It maps a grain's */
/* orientation and the load state to the elastic energy density and the       */
/* dislocation energy of Eq. (4) that the crystal plasticity of Sec. 2 would   */
/* produce, so the driving field can be refreshed per grain.                   */
/* Parameters: one FP32 device buffer of hp_mlp_param_count() floats, in the   */
/* order W1[64][11], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[2][64],*/
/* b4[2] (W_l maps layer l-1 to layer l; rows are output features).            */
/* Inputs X: device float[M][11]; targets T and outputs Y: device float[M][2]. */
/* ------------------------------------------------------------------------ */
HP_API int hp_mlp_param_count(int64_t* n);
/* Y = MLP(X): inputs, weights and hidden activations rounded to BF16, every sum
 * in FP32.  Asynchronous; a tensor-core wait that runs out of time is reported
 * by hp_mlp_status.                                                          */
HP_API int hp_mlp_forward(const float* params, const float* X, int64_t M, float* Y, void* stream);
/* grads (device float[param_count], overwritten) = dL/dparams and *loss (device
 * float, may be NULL) = L for L = 1/(2M) sum_rows sum_outputs (y - t)^2.      */
HP_API int hp_mlp_gradients(const float* params, const float* X, const float* T, int64_t M, float* grads,
                            float* loss, void* stream);
/* The network's activation as the kernels evaluate it, for testing: g[i] =
 * GELU(z[i]) = z Phi(z) and dg[i] = Phi(z) + z phi(z) (device float[n] each),
 * Phi through erf by Abramowitz and Stegun 7.1.26 (|error| <= 1.5e-7).       */
HP_API int hp_debug_gelu(const float* z, int64_t n, float* g, float* dg, void* stream);

/* One Adam step (Kingma & Ba) on the FP32 master weights: m, v (device float
 * [param_count]) are the moment estimates, step counts from 1.               */
HP_API int hp_mlp_adam(float* params, const float* grads, float* m, float* v, int32_t step, float lr, float beta1,
                       float beta2, float eps, void* stream);
/* Synchronous: HP_ERR_TIMEOUT if any surrogate kernel since the last call gave
 * up waiting for its tensor-core operations (bounded, about two seconds);
 * clears the flag.  *timed_out = 1: the block then waited up to four more
 * limits for the pending commit before freeing its tensor memory; 2: that
 * drain ran out too and the context should not be trusted.                  */
HP_API int hp_mlp_status(int32_t* timed_out);

/* Fixed normalisation of the surrogate's inputs and targets.                  */
typedef struct {
    float stress; /* MPa per unit input (sample-frame stress components)       */
    float strain; /* slip per unit input (average accumulated slip)            */
    float w;      /* MJ/m^3 per unit of the first output (elastic energy)      */
    float erho;   /* MJ/m^3 per unit of the second output (dislocation energy) */
} hp_sur_scales;

/* Training data from the crystal plasticity itself (Sec. 2): n_orient
 * orientations (device float[4 n_orient]) each followed through load
 * increments t = 1..n_incr (Eq. (3)) in K stochastic histories (K material
 * points, Philox counters n_orient*K apart).  After increment t, with
 * sigma_hat(t) = population average of the sample-frame stress R sigma R^T and
 * gamma_hat(t) = average slip, sample o*n_incr + (t-1) is (orientation-major,
 * so any contiguous run of rows covers whole orientations at every increment)
 *   X = (f(q_o), sigma_hat(t)/stress, gamma_hat(t)/strain)     (device float[.][11])
 * where f(q) encodes the orientation by four cubic invariants of the loading
 * axis d = R(q)^T e_x: |d| sorted in decreasing order and
 * d1^2 d2^2 + d2^2 d3^2 + d3^2 d1^2 (the Taylor strain is axisymmetric about x,
 * so only d, modulo the cubic symmetry, matters)
 *   Y = (<w>_K / w, <E_rho>_K / erho)                           (device float[.][2])
 * load_out (device float[n_incr][7], may be NULL) receives (sigma_hat, gamma_hat)
 * unscaled.  Allocates its own work buffers.                                 */
HP_API int hp_sur_generate(const hp_cp_params* prm, uint64_t seed, const float* quat, int32_t n_orient, int32_t K,
                           int32_t n_incr, const hp_sur_scales* sc, float* X, float* Y, float* load_out,
                           void* stream);
/* Training of the surrogate on data of hp_sur_generate: `steps` Adam steps
 * (hp_mlp_adam, step numbers step0 + 1 .. step0 + steps) on the loss of
 * hp_mlp_gradients over minibatches of `batch` rows (rounded down to whole
 * groups of `group` consecutive rows; 0 = every row) taken in turn from the
 * start of X (device float[M][11]) and Y (device float[M][2]); the learning
 * rate decays from lr to lr_floor * lr by a half cosine over the run:
 *   lr_t = lr (lr_floor + (1 - lr_floor) (1 + cos(pi t / steps)) / 2).
 * params, m, v: device float[hp_mlp_param_count()], updated in place.  loss
 * (device float, may be NULL) receives the last minibatch loss; with
 * log_every > 0 the loss after every log_every-th step is also copied to the
 * host array loss_log[steps / log_every] (copied after the run).
 * The whole run is one cooperative launch when every CTA of the gradient kernel
 * can be resident (one per SM): a grid barrier separates each step's gradients
 * from its update.  Work on other streams that keeps SMs busy can hold CTAs
 * back; a barrier then gives up after about two seconds, the run stops early and
 * hp_mlp_status reports HP_ERR_TIMEOUT.  When the CTAs cannot all be resident
 * the steps run as two launches each instead (same arithmetic).  Allocates its
 * work buffers (gradient slots, packed weights, the schedule) for the duration
 * of the call and synchronises the stream before returning.                  */
typedef struct {
    int32_t steps;    /* Adam steps                                           */
    int64_t batch;    /* rows per minibatch (0 = all rows)                    */
    int32_t group;    /* rows per group: minibatches hold whole groups        */
    float lr;         /* initial learning rate                                */
    float lr_floor;   /* final learning rate as a fraction of lr, in [0, 1]   */
    float beta1, beta2, eps; /* Adam constants                                */
    int32_t log_every;/* 0: no loss log                                       */
} hp_sur_train_params;
HP_API int hp_sur_train(float* params, float* m, float* v, const float* X, const float* Y, int64_t M,
                        const hp_sur_train_params* tp, int32_t step0, float* loss, float* loss_log, void* stream);

/* Per-grain driving field from the surrogate at one load state (host float[7]
 * = sigma_hat, gamma_hat): y = MLP(f(q_g), load), e_g = energy_scale (y0 w + y1 erho)
 * [J], b_g = round-half-even(256 e_g) clamped to +-2^20 into b_out (device
 * int32[G], the HP_FIELD_GRAIN table); e_out (device float[G]) may be NULL.
 * Asynchronous on `stream`; the host load vector is read before the call
 * returns and may be released at once.                                       */
HP_API int hp_sur_field(const float* params, const float* quat, int32_t G, const float* load, const hp_sur_scales* sc,
                        double energy_scale, int32_t* b_out, float* e_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HMCPOTTS_H */
