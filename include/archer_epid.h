/*
 * archer_epid.h -- C ABI of the B300 EPID transit Monte Carlo library.
 *
 * The library computes, on one GPU, the data-parallel core of the method of
 * "A GPU-based Monte Carlo framework for IMRT QA using EPID transit dosimetry"
 * (ARCHER-EPID): photons from an MLC-shaped 6 MV source (Sec. 2.1.1) are
 * transported with coupled photon/electron Monte Carlo through a CT-derived
 * voxel patient (Sec. 2.1.2) into a multi-layer EPID (Sec. 2.1.3); the energy
 * deposited in the sensitive layer is tallied per pixel and converted into a
 * detector signal with the k(t, s) table of Sec. 2.2 / Sec. 3.1 (Eq. 1, Eq. 2,
 * Table 1).
 *
 * Conventions (all entry points):
 *  - Every call returns an mc_status; no C++ exception crosses the ABI.
 *    mc_last_error() returns a description of the last failure of a context.
 *  - Pointers are plain host or device addresses as stated per argument; the
 *    caller owns every array it passes and every output buffer.  Inputs are
 *    copied, so they may be freed when the call returns (device inputs: once
 *    the stream has reached the call).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    queued on it.  mc_run (graph-driven, the default) returns without
 *    waiting for the device; every later call of the context that reads or
 *    changes its device state is ordered after that run (on its own stream by
 *    an event wait, or by waiting on the host where it says so).  Calls that
 *    write host outputs return once their results are there.
 *  - Units: cm, MeV, g/cm^3; doses in Gy per source history.
 *  - Arrays are row-major, last index fastest: CT [nz][ny][nx], EPID images
 *    [npy][npx], tallies [B][npy][npx], k-table [ns][nt].
 *  - A context is bound to one device and is not thread-safe; use one context
 *    per host thread.
 */
#ifndef ARCHER_EPID_H
#define ARCHER_EPID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mc_status {
    MC_OK = 0,
    MC_ERR_ARG = 1,        /* invalid argument (null pointer, size, range, order of calls) */
    MC_ERR_CUDA = 2,       /* a CUDA runtime call failed; see mc_last_error */
    MC_ERR_OOM = 3,        /* device allocation failed */
    MC_ERR_STATE = 4,      /* call out of order (e.g. mc_run before mc_set_field) */
    MC_ERR_TIMEOUT = 5,    /* a bounded device wait gave up */
    MC_ERR_CANCELLED = 6,  /* mc_cancel() stopped the run between waves */
    MC_ERR_NUMERIC = 7,    /* non-finite value detected */
    MC_ERR_OVERFLOW = 8    /* a particle bank filled; the run's energy balance is incomplete */
} mc_status;

/* Material ids (compositions are the library's stated readings; the paper
 * names the materials of Sec. 2.1.2 / Sec. 2.1.3 without giving data). */
enum {
    MC_MAT_AIR = 0, MC_MAT_LUNG = 1, MC_MAT_WATER = 2, MC_MAT_BONE = 3,
    MC_MAT_CU = 4, MC_MAT_GD2O2S = 5, MC_MAT_SI = 6, MC_NUM_MATERIALS = 7
};

#define MC_MAX_LAYERS 8
#define MC_NUM_COUNTERS 20

/* Event counters, in the order of mc_run_stats.counters. */
enum {
    MC_CNT_FLIGHTS_CT = 0, MC_CNT_REAL_CT, MC_CNT_COMPTON, MC_CNT_PHOTO, MC_CNT_PAIR,
    MC_CNT_ESTEPS_CT, MC_CNT_ESTEPS_EPID, MC_CNT_MOLLER, MC_CNT_BREM, MC_CNT_PRIMARIES_AT_EPID,
    MC_CNT_UNCOLLIDED_AT_EPID, MC_CNT_LOST, MC_CNT_FLIGHTS_EPID, MC_CNT_ELECTRONS, MC_CNT_POSITRONS,
    MC_CNT_SECONDARY_PHOTONS,
    /* execution: warp iterations and live lanes summed over them, for the CT
     * photon and CT electron kernels (live / (32 iterations) = lane utilisation) */
    MC_CNT_WARP_ITERS_PHOTON_CT, MC_CNT_LIVE_LANES_PHOTON_CT, MC_CNT_WARP_ITERS_ELECTRON_CT,
    MC_CNT_LIVE_LANES_ELECTRON_CT
};

/* Transport and execution settings.  Physics fields follow Sec. 2.1.2
 * (10 keV photon and 200 keV electron cutoffs, Class II condensed history);
 * the others are stated readings.  Fill with mc_config_default() first. */
typedef struct mc_config {
    int coupled;                  /* 1: transport electrons/positrons; 0: deposit them where created */
    double e_max_mev;             /* 6 MV spectrum end point: E = e_max * Beta(3/2, 7/2) */
    double mono_energy_mev;       /* > 0: monoenergetic source instead of the spectrum */
    double photon_cutoff_mev;     /* 0.01 */
    double electron_cutoff_mev;   /* 0.2 */
    double wcc_mev;               /* hard Moller threshold, 0.2 */
    double wcb_mev;               /* hard bremsstrahlung threshold, 0.01 */
    double step_fraction;         /* largest CSDA energy-loss fraction per electron step, 0.05 */
    int n_batches;                /* B sub-tallies (history id mod B) for the uncertainty, 16 */
    int max_steps;                /* per-particle step cap; beyond it the energy is counted as lost */
    int block_size;               /* threads per CTA of the transport kernels (multiple of 32), 0 = 256 */
    int ctas_per_sm;              /* resident CTAs per SM for the persistent kernels, 0 = occupancy limit */
    uint32_t bank_capacity;       /* particles per bank, 0 = 1<<23 */
    uint32_t primaries_per_wave;  /* new histories per transport wave, 0 = bank_capacity / 4; a wave admits
                                     no more than half a bank or the room left in the CT-photon bank */
    int time_kernels;             /* 1: time every transport launch with CUDA events (mc_run_stats.kernel_ms);
                                     needs the host-driven loop, so mc_run then waits for the device */
    int use_graph;                /* 1 (default): each run is one CUDA-graph launch whose waves loop on the
                                     device (a conditional while-node) and mc_run does not wait for it;
                                     0: waves are driven from the host, which reads the run control after
                                     every wave (mc_run then waits, and mc_cancel can stop it) */
    int regs_variant[4];          /* per transport kernel (CT photons, CT electrons, EPID photons, EPID
                                     electrons): build for 2, 3 or 4 CTAs of 256 threads per SM
                                     (register caps 128 / 85 / 64); 0 = the default 4 */
    int patient_dose;             /* 1: also tally the energy deposited in every CT voxel (the patient
                                     dose of the same histories; mc_get_patient_dose) */
} mc_config;

/* EPID layer stack from the source side (Sec. 2.1.3).  The centre of the
 * sensitive layer lies on the plane at SID from the source; the pixel grid
 * (npx along beam-frame X, npy along Y, pitch at the detector plane) also
 * sets the detector's lateral extent. */
typedef struct mc_epid_desc {
    int n_layers;                         /* 1 .. MC_MAX_LAYERS */
    int material[MC_MAX_LAYERS];          /* MC_MAT_* */
    double thickness_cm[MC_MAX_LAYERS];
    double density[MC_MAX_LAYERS];
    int sensitive_layer;
    int npx, npy;
    double pitch_cm;
} mc_epid_desc;

/* One static IMRT field (Sec. 2.1.1): MLC segments at the isocentre plane.
 * Host pointers; copied by mc_set_field. */
typedef struct mc_field_desc {
    int n_segments, n_pairs;
    const double* pair_edges_cm;  /* [n_pairs + 1] leaf-pair boundaries along Y, increasing */
    const double* leaves_cm;      /* [n_segments][n_pairs][2] left/right leaf tips along X */
    const double* jaws_cm;        /* [n_segments][4] x1, x2, y1, y2 */
    const double* mu;             /* [n_segments] monitor units (>= 0, not all zero) */
    double gantry_deg;            /* rotation of source and EPID about the patient z axis */
    double sad_cm, sid_cm;
    double iso_cm[3];             /* isocentre in CT coordinates */
    int eq1_literal;              /* 0: s = 2ab/(a+b); 1: s = ab/(2(a+b)) exactly as Eq. 1 is printed */
    /* Collimation (Sec. 2.1.1 transports the beam through jaws and MLC), in
     * one of two models, inside the largest field |X|, |Y| <= 20 cm and the
     * MLC's extent.  Fluence filters on the isocentre plane: per MU the
     * fluence is (leaf factor) x (jaw factor): 1 inside the effective opening
     * of the point's leaf pair, else leaf_transmission; 1 inside the segment's
     * jaws, else jaw_transmission.  All zero: the ideal aperture.  Or slabs
     * (leaf_thickness_cm / jaw_thickness_cm below). */
    double leaf_transmission;     /* 0 <= T < 1 */
    double jaw_transmission;      /* 0 <= Tj < 1 */
    double tg_width_cm;           /* tongue and groove: within half this width of a pair boundary the
                                     opening is the intersection of both pairs' openings;
                                     0 <= w < narrowest pair */
    double leaf_gap_cm;           /* dosimetric leaf gap: an open pair's tips move apart by g/2 each
                                     (rounded leaf ends); a pair whose tips meet stays closed; 0 <= g < 2 */
    /* Collimator slabs: the leaves and jaws as laterally infinite tungsten
     * slabs (19.3 g/cm^3) of these thicknesses along the beam, the jaws' top
     * 28 cm and the leaves' top 51 cm from the source.  Either > 0 switches
     * the source to phase space 2 of Sec. 2.1.1: photons of the open-beam
     * source are drawn uniformly over the 40 x 40 cm field (segments by MU)
     * until one leaves the slabs its ray crosses (a jaw slab outside the
     * segment's jaws, a leaf slab outside its pair's effective opening), with
     * Compton scattering in the tungsten and photoelectric and pair
     * absorption there; that photon, from the bottom of its last slab, is the
     * history.  Then both transmissions above must be 0.  A slab of
     * thickness 0 is ideal (opaque). */
    double leaf_thickness_cm;     /* 0 <= t <= 20 */
    double jaw_thickness_cm;      /* 0 <= t < 23 */
} mc_field_desc;

/* k(t, s) table of Sec. 3.1 (Eq. 2, Table 1): k[is * nt + it] on strictly
 * increasing node axes, bilinear inside and clamped outside.  Host pointers. */
typedef struct mc_lut_desc {
    int nt, ns;                   /* 2 .. 1024 each */
    const double* t_nodes;        /* radiological thickness, cm */
    const double* s_nodes;        /* equivalent square field size, cm */
    const double* k;              /* [ns][nt] */
    double k_scale;               /* signal = k_scale * k(t, s) * dose */
    double t_offset_cm;           /* added to every ray sum (e.g. a couch) */
} mc_lut_desc;

/* Cumulative results since the last mc_set_field / mc_reset_tally. */
typedef struct mc_run_stats {
    uint64_t histories;
    double e_src_mev, e_ct_mev, e_epid_mev[MC_MAX_LAYERS], e_esc_mev, e_lost_mev;
    uint64_t counters[MC_NUM_COUNTERS];
    int waves;                    /* transport waves of the last mc_run */
    uint32_t error_flags;         /* device-side error bits of the last mc_run */
    double gpu_ms;                /* device time of the last mc_run (CUDA events) */
    double kernel_ms[4];          /* with time_kernels: summed time per transport kernel of the last mc_run
                                     (CT photons, CT electrons, EPID photons, EPID electrons) */
    uint32_t kernel_launches[4];  /* launches per transport kernel in the last mc_run */
    uint32_t launches;            /* all kernel launches of the last mc_run */
} mc_run_stats;

typedef struct mc_ctx mc_ctx;

/* Defaults stated above. */
void mc_config_default(mc_config* cfg);

/* Creates a context on `device`, allocating its particle banks and tables.
 * cfg may be NULL (defaults).  *out is NULL on failure. */
mc_status mc_create(const mc_config* cfg, int device, mc_ctx** out);

/* Frees every device and host allocation of ctx (NULL is a no-op). */
mc_status mc_destroy(mc_ctx* ctx);

/* CT set-up (Sec. 2.1.2, HU-to-density curve): copies the int16 HU volume
 * [nz][ny][nx] (host pointer, or device pointer when hu_on_device != 0) and
 * converts it on the GPU to per-voxel density; material follows from the
 * density thresholds.  vox_cm: voxel size, origin_cm: lower corner of the box.
 * Also takes the EPID stack.  Invalidates any field set before. */
mc_status mc_init_geometry(mc_ctx* ctx, const int16_t* hu, int nx, int ny, int nz, const double vox_cm[3],
                           const double origin_cm[3], const mc_epid_desc* epid, int hu_on_device,
                           void* stream);

/* The field of Sec. 2.1.1 (MLC segments, jaws, MU weights, gantry angle) and
 * the correction inputs of Sec. 2.2: builds the source's aperture table, the
 * radiological thickness map (Sec. 2.2 item 1: a ray sum of density from the
 * source to every pixel centre, FP64 accumulation), the field size of Eq. 1
 * (on the bounding rectangle of the union of open apertures) and uploads the
 * k-table of Sec. 3.1.  Resets the tally.  lut may be NULL (then
 * mc_get_epid_image is unavailable).  Queued on `stream` without waiting for
 * the device: host data goes through pinned staging, and the device buffers
 * of the previous field are reused when large enough (when one must grow,
 * the call first waits for a pending run). */
mc_status mc_set_field(mc_ctx* ctx, const mc_field_desc* field, const mc_lut_desc* lut, void* stream);

/* The Monte Carlo transport of Sec. 2.1: n_histories photons of every field
 * set on the context from the MLC-shaped source (Sec. 2.1.1) through the CT
 * patient (Sec. 2.1.2: photoelectric, Compton, pair; Class II condensed
 * history electrons) into the EPID layer stack (Sec. 2.1.3), the energy left
 * in the sensitive layer added to the per-pixel tally.  History ids continue
 * from the previous run, so repeated calls equal one longer run; Philox is
 * keyed by seed.
 * With use_graph (the default) and no time_kernels the run is queued on
 * `stream` as one graph launch and the call returns without waiting; the
 * tally and the stats are valid once the stream has passed the run.  A
 * non-NULL `stats` makes the call wait and fill it.  Device-side failures
 * (MC_ERR_OVERFLOW, MC_ERR_TIMEOUT) of a run that did not wait are returned
 * by the next mc_get_stats, mc_run, mc_set_field that replaces buffers, or
 * mc_init_geometry.  With use_graph = 0 or time_kernels the call waits. */
mc_status mc_run(mc_ctx* ctx, uint64_t n_histories, uint64_t seed, void* stream, mc_run_stats* stats);

/* Batching (several static fields of one plan on one phantom, Sec. 2.3's 25
 * IMRT fields): sets n_fields fields (1 .. 256) at once, each with its own
 * source, beam frame (gantry angle), radiological-thickness map and Eq. 1
 * field size, sharing the CT, the EPID and the k-table.  Each field keeps its
 * own tally; field f draws from the same random streams as a single-field run
 * whose history ids start at f * 2^40 (so a batch equals its fields run one
 * by one).  Resets the tallies. */
mc_status mc_set_fields(mc_ctx* ctx, const mc_field_desc* fields, int n_fields, const mc_lut_desc* lut,
                        void* stream);

/* Transports n_histories[f] histories of every field f in one wave sequence
 * (one graph launch with use_graph), so fields of uneven sizes share the GPU.
 * Waits for the device as mc_run does. */
mc_status mc_run_batch(mc_ctx* ctx, const uint64_t* n_histories, uint64_t seed, void* stream,
                       mc_run_stats* stats);

/* Per-field read-outs: as mc_get_dose, mc_get_epid_image, mc_get_tmap and
 * mc_field_size for field `field` (0 .. n_fields-1). */
mc_status mc_get_field_dose(mc_ctx* ctx, int field, double* dose, double* sigma, double* u_out, int on_device,
                            void* stream);
mc_status mc_get_field_image(mc_ctx* ctx, int field, float* signal, int on_device, void* stream);
mc_status mc_get_field_tmap(mc_ctx* ctx, int field, double* t, int on_device, void* stream);
mc_status mc_get_field_size(mc_ctx* ctx, int field, double* s, double* a, double* b);

/* The per-pixel EPID dose and its statistical uncertainty (Sec. 2.3: images
 * of 1e9 histories at < 1 %; the paper does not define the figure, this
 * library reports the batch estimate), field 0: per-history dose (Gy) in
 * the sensitive layer and its batch standard error over B sub-tallies,
 * [npy][npx] doubles (host or device per on_device); sigma may be NULL.
 * u_out (host, may be NULL) receives the mean relative uncertainty over
 * pixels above half the maximum dose.  With on_device and no u_out the work
 * is queued on `stream` and the call does not wait. */
mc_status mc_get_dose(mc_ctx* ctx, double* dose, double* sigma, double* u_out, int on_device, void* stream);

/* The field's source fluence on the EPID grid: the probability density
 * (cm^-2 at the isocentre plane) of a history's source ray crossing that
 * plane at each pixel centre scaled by SAD / SID -- the MLC- and
 * jaw-modulated source of Sec. 2.1.1 that mc_run samples (MU weights, leaf
 * and jaw transmission, tongue and groove, leaf gap; with collimator slabs,
 * the rays before the slabs).  It integrates to 1 over the isocentre plane.
 * Segments add their densities with atomics, so repeated calls agree up to
 * the order of those sums (~1e-16 relative).
 * F: [npy][npx] doubles, host or device per on_device.  With on_device the
 * work is queued on `stream` and the call does not wait. */
mc_status mc_get_field_fluence(mc_ctx* ctx, int field, double* F, int on_device, void* stream);

/* Mean per-history dose (Gy) over the pixel rectangle [ix0, ix1) x [iy0, iy1)
 * of field `field` and the batch standard error of that mean (the central
 * 1 cm x 1 cm region of the Sec. 2.2 calibration, whose signal enters Eq. 2;
 * uncertainty as for mc_get_dose, Sec. 2.3): mean = sum of the region's
 * deposits / (N x pixels), the error from the B per-batch region means.
 * mean and sigma are host doubles (sigma may be NULL).  Errors: MC_ERR_ARG
 * for an empty rectangle or one not inside the image, MC_ERR_STATE before
 * any history.  Waits for the device. */
mc_status mc_get_region_dose(mc_ctx* ctx, int field, int ix0, int ix1, int iy0, int iy1, double* mean,
                             double* sigma, void* stream);

/* The k(t, s) correction (Sec. 3.1, field 0): signal = k_scale * k(t, s) * dose per pixel, float32
 * [npy][npx] (host or device per on_device). */
mc_status mc_get_epid_image(mc_ctx* ctx, float* signal, int on_device, void* stream);

/* The radiological thickness map t (cm, FP64) of field 0. */
mc_status mc_get_tmap(mc_ctx* ctx, double* t, int on_device, void* stream);

/* Raw integer sub-tallies [n_fields][B][npy][npx], unit 2^-8 eV. */
mc_status mc_get_tally(mc_ctx* ctx, uint64_t* tally, int on_device, void* stream);

/* Equivalent square s (Eq. 1 reading) and bounding rectangle sides a, b (cm) of field 0. */
mc_status mc_field_size(mc_ctx* ctx, double* s, double* a, double* b);

/* Plan image (VMAT arcs and multi-field plans): with the fields of a batch
 * as control points, dose = sum_f w_f D_f and signal = sum_f w_f k(t_f, s_f)
 * D_f over the fields, D_f the per-history dose of field f, t_f its
 * radiological-thickness map and s_f its Eq. 1 size -- what an EPID
 * integrating over the arc records per unit weight.  weights: host array of
 * n_fields (e.g. MU fractions) or NULL for equal weights 1/n_fields.  dose
 * and signal: [npy][npx] doubles (host or device per on_device); either may
 * be NULL; signal needs the k-table. */
mc_status mc_get_plan_image(mc_ctx* ctx, const double* weights, double* dose, double* signal, int on_device,
                            void* stream);

/* Bilinear resampling of an image between pixel grids centred on the same
 * axis (pixel centres at ((i + 1/2) - n/2) pitch; the border value is held
 * beyond the outer centres), e.g. a 2.5 mm dose image onto the detector's
 * 1190 x 1190 grid at 0.336 mm (Sec. 2.3).  src [sny][snx], dst [dny][dnx]:
 * device doubles.  Synchronizes `stream`. */
mc_status mc_resample_image(const double* src, int snx, int sny, double src_pitch, double* dst, int dnx, int dny,
                            double dst_pitch, void* stream);

/* Patient dose (the dose engine the method builds on, Sec. 2.1):
 * with mc_config.patient_dose, every energy deposit in the CT also goes, in
 * the same 2^-8 eV units, to the voxel the particle is in, for all fields
 * and runs since the tally was last reset.  dose (host or device per
 * on_device) receives [nz][ny][nx] doubles: Gy per source history =
 * E / (rho V) / N, rho from the HU curve, V the voxel volume, N the histories
 * of all fields.  MC_ERR_STATE when patient dose is off or nothing has run. */
mc_status mc_get_patient_dose(mc_ctx* ctx, double* dose, int on_device, void* stream);

/* Cumulative statistics (energy balance from the fixed-point counters).
 * Waits for a pending run and returns its device-side outcome (MC_OK,
 * MC_ERR_OVERFLOW or MC_ERR_TIMEOUT), with the stats filled either way. */
mc_status mc_get_stats(mc_ctx* ctx, mc_run_stats* stats);

/* Clears tally, counters and the history id sequence. */
mc_status mc_reset_tally(mc_ctx* ctx, void* stream);

/* Checkpoint / resume: the state is the sub-tallies, counters and next history
 * id.  mc_state_size gives the byte size; get/set copy it to/from a host
 * buffer.  Because the random streams are keyed by history id, a resumed run
 * is bitwise identical to an uninterrupted one. */
mc_status mc_state_size(mc_ctx* ctx, size_t* bytes);
mc_status mc_get_state(mc_ctx* ctx, void* host_buf, size_t bytes, void* stream);
mc_status mc_set_state(mc_ctx* ctx, const void* host_buf, size_t bytes, void* stream);

/* Sets the id of the next history of every field (sharding: rank r of R running n histories
 * each starts at r * n, and the union of the shards equals one run of R * n
 * histories).  Does not clear the tally. */
mc_status mc_set_history_base(mc_ctx* ctx, uint64_t next_history);

/* Requests that a host-driven mc_run (use_graph = 0) running on another host
 * thread stop after its current wave (it then returns MC_ERR_CANCELLED).  A
 * graph-driven run loops on the device and runs to its end. */
mc_status mc_cancel(mc_ctx* ctx);

/* Global gamma index (Low et al. 1998), the image comparison of Sec. 2.3.3:
 * for each pixel of the reference image `ref` at or above threshold * max(ref),
 * gamma = min over offsets r (a square sub-grid of step step_mm within
 * radius_mm) of sqrt(|r|^2 / dta_mm^2 + (ev(x + r) - ref(x))^2 / (dd_frac *
 * max(ref))^2), with `ev` bilinearly interpolated and clamped at the border.
 * ref, ev: device double [ny][nx] (non-negative), pixel pitch pixel_mm;
 * gamma: device double [ny][nx] (NaN below the threshold) or NULL;
 * pass_rate (host) receives the fraction of evaluated pixels with gamma <= 1
 * (1 if none is evaluated).  step_mm <= 0 selects min(pixel_mm, dta_mm / 10),
 * radius_mm <= 0 selects 3 dta_mm.  Synchronizes `stream`. */
mc_status mc_gamma(const double* ref, const double* ev, int nx, int ny, double pixel_mm, double dd_frac,
                   double dta_mm, double threshold, double step_mm, double radius_mm, double* gamma,
                   double* pass_rate, void* stream);

/* Dose statistics without any device allocation.  The paper has no
 * counterpart: this serves callers that may not allocate device memory once
 * they are running, such as a QA service whose framework allocator has
 * already reserved the GPU's memory, or medical software whose rules forbid
 * run-time allocation because it can fail or stall unpredictably.
 *
 * Computes what mc_get_dose computes (per-history dose in Gy, its batch
 * standard error and the mean relative uncertainty over pixels above half the
 * maximum) from a tally the caller holds: tally is a device array
 * [n_batches][npy][npx] of 2^-8 eV units (as mc_get_tally writes it) for
 * history ids 0 .. n_histories-1; pixel_mass_kg is the mass of one pixel of
 * the sensitive layer.  dose and sigma (sigma may be NULL) are device arrays
 * [npy][npx]; u (device, one double, may be NULL; needs sigma) receives the
 * relative uncertainty.  The work is queued on `stream`; nothing is copied to
 * the host and nothing is allocated or freed.
 *
 * Limits: at most 4,194,304 pixels (2048 x 2048) and 1024 batches; larger
 * inputs return MC_ERR_ARG (and a message on stderr), and so does
 * n_histories < n_batches (a batch without histories has no mean).  Its
 * scratch is a 205,056-byte array inside the library that every GPU loading
 * the library keeps until the process exits.  The first call on a device
 * looks up that array's device address, so make it before capturing the
 * stream; the address is kept for the life of the process, so do not call
 * this again after cudaDeviceReset (or another destruction of the device's
 * primary context).  All calls
 * share the array: calls whose work overlaps on the GPU (two streams, or two
 * host threads) race and give wrong results; serialize them.  Call it with the
 * device that holds `tally` current. */
mc_status mc_dose_stats_noalloc(const uint64_t* tally, int npx, int npy, int n_batches, uint64_t n_histories,
                                double pixel_mass_kg, double* dose, double* sigma, double* u, void* stream);

const char* mc_last_error(const mc_ctx* ctx);
const char* mc_status_string(mc_status s);

/* Diagnostic: Philox4x32-10 (Salmon et al., SC'11) on the GPU.  in: device
 * [n][6] uint32 (ctr0..3, key0, key1), out: device [n][4]. */
mc_status mc_test_philox(const uint32_t* in, uint32_t* out, int n, void* stream);

/* Diagnostic: the first n uniforms of the draw stream of particle (hist, ord)
 * under seed, as the transport kernels draw them.  out: device float [n]. */
mc_status mc_test_uniforms(uint64_t seed, uint64_t hist, uint32_t ord, int n, float* out, void* stream);

/* Measured arithmetic peaks of this GPU: the denominators of the transport
 * kernels' ALU roofline.  Each figure is the best of `repeats` launches of a
 * full-occupancy kernel of independent dependency chains of one instruction
 * class, counted from its source:
 *   ffma_tflops   FP32 fused multiply-adds (2 flops each), scalar form
 *   ffma2_tflops  FP32 fused multiply-adds issued as fma.rn.f32x2 pairs
 *   mufu_tops     ex2.approx / lg2.approx results, T ops/s
 *   int_tinst     32-bit integer xor and add, T thread-instructions/s
 *   mix_tinst     FP32 FMA and integer ops interleaved, T thread-instructions/s
 *   ms_total      summed best times of the five probes
 * Takes about 0.1 s on device `device`; allocates and frees its own buffers.
 * MC_ERR_ARG for a null result, repeats outside [1, 100] or a bad device. */
typedef struct mc_alu_peaks {
    double ffma_tflops;
    double ffma2_tflops;
    double mufu_tops;
    double int_tinst;
    double mix_tinst;
    double ms_total;
    int32_t sm_count;
    int32_t _pad;
} mc_alu_peaks;

mc_status mc_probe_alu_peaks(int device, int repeats, mc_alu_peaks* res);

#ifdef __cplusplus
}
#endif
#endif /* ARCHER_EPID_H */
