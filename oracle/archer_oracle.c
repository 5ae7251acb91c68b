/*
 * FP64 CPU oracle for the EPID transit Monte Carlo path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path: every formula below is
 * evaluated directly in double precision from the written model, with no
 * tabulation, blocking or reordering beyond what the model states.
 *
 * What it computes (paper, Sec. 2.1): photons from an MLC-shaped point source
 * (Sec. 2.1.1; the paper's phase-space source is replaced by an ideal aperture)
 * are transported through a CT-derived voxel patient (Sec. 2.1.2: photoelectric,
 * Compton, pair production; Class II condensed-history electrons with hard
 * collisions and CSDA soft losses; cutoffs 10 keV photons / 200 keV electrons)
 * into a multi-layer EPID slab (Sec. 2.1.3) whose sensitive-layer energy is
 * tallied per pixel.  The paper gives the model class but no cross sections;
 * the parameterised fits, the HU curve and the sampling algorithms below are
 * the readings of the paper this project states, with the draw order fixed so
 * that a second implementation fed the same Philox keys replays each history.
 *
 * Parity pins: each sampler and cross section has an external check in the
 * CPU test suite (closed forms, numerical integration, brute-force
 * enumeration), and the transport loop itself is pinned through orc_pencil
 * (the loop of orc_run with one fixed primary and a recording probe): CSDA
 * track length and depth profile, Lewis' mean stopping depth, the hard-event
 * survival law, EPID layer transmission, pixel mapping, pair and annihilation
 * and interaction kinematics.  The absolute values of the builder's
 * photoelectric, pair and bremsstrahlung fits are model definitions with no
 * external data to compare against ("parity unpinned" for their magnitudes;
 * their structure is pinned).
 */
#include <math.h>
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_PI 3.14159265358979323846
#define O_RE 2.8179403262e-13      /* classical electron radius, cm */
#define O_MC2 0.51099895           /* electron rest energy, MeV */
#define O_NA 6.02214076e23         /* Avogadro, 1/mol */
#define O_ALPHA (1.0 / 137.035999084)
#define O_PE_A 4.56e-33            /* photoelectric fit: a Z^4.5 E^-3.2, cm^2 (E in MeV) */
#define O_PE_N 4.5
#define O_PE_P 3.2
#define O_GD_EK 0.05024            /* Gd K edge, MeV */
#define O_GD_JUMP 5.3              /* Gd K-edge jump ratio */
#define O_W_EK 0.069525            /* W K edge, MeV */
#define O_W_JUMP 4.6               /* W K-edge jump ratio */
#define O_W_RHO 19.3               /* tungsten collimator density, g/cm^3 */
#define O_JAW_TOP 28.0             /* jaw slab top, cm from the source */
#define O_MLC_TOP 51.0             /* MLC slab top, cm from the source */
#define O_MAT_W 7
#define O_PAIR_C 2.57e-27          /* pair fit: C Z(Z+1) (1-2mc^2/E)^4, cm^2 */
#define O_BREM_B 4.65e-27          /* bremsstrahlung fit: dsigma/dk = B Z(Z+1)/k, cm^2 */
#define O_ES 21.2                  /* Rossi scattering energy, MeV */
#define O_TSTOP 1e-6               /* an electron stops once T <= cutoff + this, MeV */
#define O_NMAT 8
#define O_MAXL 8
#define O_HOM_R 2                  /* half-width of a homogeneous voxel's neighbourhood, voxels */
#define O_HOM_SPAN 200             /* largest HU span within a homogeneous neighbourhood */

/* ------------------------------------------------------------------------ */
/* Materials: elemental mass fractions and mean excitation energies.         */
/* ------------------------------------------------------------------------ */
typedef struct { int Z; double A; double w; } o_elem;
typedef struct { int n; o_elem e[10]; double I_eV; } o_matdef;

static const o_matdef O_MATS[O_NMAT] = {
    /* 0 dry air */
    {4, {{7, 14.007, 0.755268}, {8, 15.999, 0.231781}, {18, 39.948, 0.012827}, {6, 12.011, 0.000124}}, 85.7},
    /* 1 lung (ICRU-44 composition) */
    {9, {{1, 1.008, 0.103}, {6, 12.011, 0.105}, {7, 14.007, 0.031}, {8, 15.999, 0.749}, {11, 22.990, 0.002},
         {15, 30.974, 0.002}, {16, 32.06, 0.003}, {17, 35.45, 0.003}, {19, 39.098, 0.002}}, 75.3},
    /* 2 water / soft tissue */
    {2, {{1, 1.008, 0.111894}, {8, 15.999, 0.888106}}, 75.0},
    /* 3 cortical bone (ICRU-44 composition) */
    {9, {{1, 1.008, 0.034}, {6, 12.011, 0.155}, {7, 14.007, 0.042}, {8, 15.999, 0.435}, {11, 22.990, 0.001},
         {12, 24.305, 0.002}, {15, 30.974, 0.103}, {16, 32.06, 0.003}, {20, 40.078, 0.225}}, 106.4},
    /* 4 copper */
    {1, {{29, 63.546, 1.0}}, 322.0},
    /* 5 Gd2O2S, mass fractions from molar masses */
    {3, {{64, 157.25, 0.830790}, {8, 15.999, 0.084524}, {16, 32.06, 0.084686}}, 437.0},
    /* 6 amorphous silicon */
    {1, {{14, 28.085, 1.0}}, 173.0},
    /* 7 tungsten (collimator slabs; photons only) */
    {1, {{74, 183.84, 1.0}}, 727.0},
};

/* ------------------------------------------------------------------------ */
/* Photon cross sections, cm^2/g.                                            */
/* ------------------------------------------------------------------------ */

/* Klein-Nishina total cross section per free electron, cm^2 (closed form). */
double orc_sigma_kn(double E) {
    double k = E / O_MC2;
    double a = 1.0 + 2.0 * k;
    double L = log(a);
    double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - L / k);
    double t2 = L / (2.0 * k);
    double t3 = (1.0 + 3.0 * k) / (a * a);
    return 2.0 * O_PI * O_RE * O_RE * (t1 + t2 - t3);
}

/* Per-gram partial attenuation coefficients of material m at photon energy E.
 * out[0] Compton, out[1] photoelectric, out[2] pair. */
void orc_mu_photon(int m, double E, double out[3]) {
    const o_matdef* md = &O_MATS[m];
    double zA = 0.0, pe = 0.0, zz = 0.0;
    for (int i = 0; i < md->n; i++) {
        const o_elem* el = &md->e[i];
        zA += el->w * el->Z / el->A;
        double pz = el->w / el->A * pow((double)el->Z, O_PE_N);
        if (el->Z == 64 && E < O_GD_EK) pz /= O_GD_JUMP;
        if (el->Z == 74 && E < O_W_EK) pz /= O_W_JUMP;
        pe += pz;
        zz += el->w * el->Z * (el->Z + 1.0) / el->A;
    }
    out[0] = O_NA * zA * orc_sigma_kn(E);
    out[1] = O_NA * O_PE_A * pow(E, -O_PE_P) * pe;
    double thr = 2.0 * O_MC2;
    out[2] = (E > thr) ? O_NA * O_PAIR_C * zz * pow(1.0 - thr / E, 4.0) : 0.0;
}

static double mu_total(int m, double E) {
    double p[3];
    orc_mu_photon(m, E, p);
    return p[0] + p[1] + p[2];
}

/* ------------------------------------------------------------------------ */
/* Electron quantities (per gram).                                           */
/* ------------------------------------------------------------------------ */
static double mat_zA(int m) {
    double s = 0.0;
    for (int i = 0; i < O_MATS[m].n; i++) s += O_MATS[m].e[i].w * O_MATS[m].e[i].Z / O_MATS[m].e[i].A;
    return s;
}
static double mat_zz(int m) {
    double s = 0.0;
    for (int i = 0; i < O_MATS[m].n; i++) {
        const o_elem* el = &O_MATS[m].e[i];
        s += el->w * el->Z * (el->Z + 1.0) / el->A;
    }
    return s;
}
/* inverse radiation length, cm^2/g: 4 alpha r_e^2 N_A sum (w/A) Z(Z+1) ln(183 Z^-1/3) */
static double mat_x0inv(int m) {
    double s = 0.0;
    for (int i = 0; i < O_MATS[m].n; i++) {
        const o_elem* el = &O_MATS[m].e[i];
        s += el->w / el->A * el->Z * (el->Z + 1.0) * log(183.0 * pow((double)el->Z, -1.0 / 3.0));
    }
    return 4.0 * O_ALPHA * O_RE * O_RE * O_NA * s;
}

/* Restricted collision stopping power (Bethe, soft Moller losses below wcc,
 * no density effect), MeV cm^2/g. */
double orc_lcol(int m, double T, double wcc) {
    double tau = T / O_MC2, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double D = fmin(wcc, 0.5 * T) / O_MC2;
    double Imc = O_MATS[m].I_eV * 1e-6 / O_MC2;
    double F = -1.0 - b2 + log((tau - D) * D) + tau / (tau - D)
               + (0.5 * D * D + (2.0 * tau + 1.0) * log(1.0 - D / tau)) / (g * g);
    double pref = 2.0 * O_PI * O_RE * O_RE * O_MC2 * O_NA * mat_zA(m) / b2;
    return pref * (log(2.0 * (tau + 2.0) / (Imc * Imc)) + F);
}

/* Bremsstrahlung strength A_m = N_A B sum (w/A) Z(Z+1), cm^2/g. */
static double brem_A(int m) { return O_NA * O_BREM_B * mat_zz(m); }

/* Soft (k < wcb) radiative stopping power, MeV cm^2/g. */
double orc_lrad_soft(int m, double T, double wcb) { return brem_A(m) * fmin(wcb, T); }

/* Hard Moller cross section (secondary above wcc), cm^2/g. */
double orc_sigma_moller(int m, double T, double wcc) {
    if (T <= 2.0 * wcc) return 0.0;
    double tau = T / O_MC2, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double ec = wcc / T, c = tau / g, bb = (2.0 * tau + 1.0) / (g * g);
    double br = 1.0 / ec - 1.0 / (1.0 - ec) + (0.5 - ec) * c * c - bb * log((1.0 - ec) / ec);
    return O_NA * mat_zA(m) * 2.0 * O_PI * O_RE * O_RE * O_MC2 / (b2 * T) * br;
}

/* Hard bremsstrahlung cross section (photon above wcb), cm^2/g. */
double orc_sigma_brem(int m, double T, double wcb) { return (T > wcb) ? brem_A(m) * log(T / wcb) : 0.0; }

/* Inverse first transport mean free path (Rossi scattering power), cm^2/g. */
double orc_lambda1_inv(int m, double T) {
    double pc2 = T * (T + 2.0 * O_MC2);
    double b2p2 = pc2 * pc2 / ((T + O_MC2) * (T + O_MC2));
    return 0.5 * O_ES * O_ES * mat_x0inv(m) / b2p2;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the per-particle    */
/* draw stream.  Draw d of particle (hist h, ordinal o) is word d mod 4 of   */
/* Philox(counter = (d div 4, o, h_lo, h_hi), key = (seed_lo, seed_hi)),     */
/* mapped to ((u >> 9) + 0.5) 2^-23, a value exact in single and double      */
/* precision and strictly inside (0, 1).  Electron steps and photon flights  */
/* start at the next multiple of 4 (rng_align).                              */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* MurmurHash3 32-bit finaliser, used to derive secondary ordinals. */
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;
    return h;
}
uint32_t orc_child_ordinal(uint32_t parent, uint32_t draws, uint32_t slot) {
    return fmix32(parent * 0x85EBCA6Bu + (draws * 8u + slot + 1u));
}

typedef struct {
    uint32_t key[2];
    uint32_t ord, hlo, hhi;
    uint32_t d;
    uint32_t cblk; int cvalid; uint32_t cbuf[4];
} o_rng;

/* Every electron step and every photon flight starts on a fresh Philox block:
 * the draw counter is rounded up to a multiple of 4. */
static void rng_align(o_rng* r) { r->d = (r->d + 3u) & ~3u; }

static double rng_u(o_rng* r) {
    uint32_t blk = r->d >> 2, w = r->d & 3u;
    if (!r->cvalid || r->cblk != blk) {
        uint32_t ctr[4] = {blk, r->ord, r->hlo, r->hhi};
        orc_philox(ctr, r->key, r->cbuf);
        r->cblk = blk; r->cvalid = 1;
    }
    r->d++;
    return ((double)(r->cbuf[w] >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* ------------------------------------------------------------------------ */
/* Samplers.                                                                  */
/* ------------------------------------------------------------------------ */

/* Source spectrum: E = Emax X, X ~ Beta(3/2, 7/2) drawn exactly as
 * G1/(G1+G2) with G1 ~ Gamma(3/2) = Exp + N^2/2 and G2 ~ Gamma(7/2) =
 * Exp+Exp+Exp + N'^2/2, the two normals from one Box-Muller pair.  Six draws
 * per attempt (u_a, u_b, u_c, u_d, u_1, u_2); attempts below the photon
 * cutoff are redrawn. */
static double sample_spectrum(o_rng* r, double emax, double ecut) {
    for (;;) {
        double ua = rng_u(r), ub = rng_u(r), uc = rng_u(r), ud = rng_u(r);
        double u1 = rng_u(r), u2 = rng_u(r);
        double L = -log(u1);
        double c = cos(2.0 * O_PI * u2);
        double g1 = -log(ua) + L * c * c;
        double g2 = -log(ub * uc * ud) + L * (1.0 - c * c);
        double E = emax * g1 / (g1 + g2);
        if (E >= ecut) return E;
    }
}

/* Klein-Nishina: composition-rejection on eps = E'/E (three draws per attempt),
 * then returns eps and cos(theta). */
static void sample_kn(o_rng* r, double E, double* eps_out, double* cos_out) {
    double k = E / O_MC2;
    double e0 = 1.0 / (1.0 + 2.0 * k);
    double a1 = log(1.0 + 2.0 * k);
    double a2 = 0.5 * (1.0 - e0 * e0);
    for (;;) {
        double r1 = rng_u(r), r2 = rng_u(r), r3 = rng_u(r);
        double eps;
        if (r1 * (a1 + a2) < a1) eps = exp(-a1 * r2);
        else eps = sqrt(e0 * e0 + (1.0 - e0 * e0) * r2);
        double t = (1.0 - eps) / (k * eps);
        double s2 = t * (2.0 - t);
        double g = 1.0 - eps * s2 / (1.0 + eps * eps);
        if (r3 < g) { *eps_out = eps; *cos_out = 1.0 - t; return; }
    }
}

/* Moller: eps = W/T on [wcc/T, 1/2] from 1/eps^2, rejection on the bracket. */
static double sample_moller_eps(o_rng* r, double T, double wcc) {
    double tau = T / O_MC2, g = tau + 1.0;
    double ec = wcc / T, c = tau / g, bb = (2.0 * tau + 1.0) / (g * g);
    double gmax = 2.0 - bb + 0.25 * c * c;
    for (;;) {
        double r1 = rng_u(r), r2 = rng_u(r);
        double eps = ec / (1.0 - r1 * (1.0 - 2.0 * ec));
        double x = eps / (1.0 - eps);
        double gv = 1.0 + x * x + c * c * eps * eps - bb * x;
        if (r2 * gmax < gv) return eps;
    }
}

/* Mean of mu=(1-cos)/2 under the screened-Rutherford law with screening A. */
static double wentzel_mean(double A) {
    if (A > 100.0) {
        double x = 1.0 / A, s = 0.0, xn = 1.0;
        for (int n = 1; n <= 10; n++) { s += ((n & 1) ? 1.0 : -1.0) * xn / (n * (n + 1.0)); xn *= x; }
        return s;
    }
    return A * ((1.0 + A) * log1p(1.0 / A) - 1.0);
}

/* Screening parameter A such that <1-cos> = 1 - exp(-G); A<0 flags isotropic. */
double orc_wentzel_A(double G) {
    if (G <= 0.0) return 0.0;
    double m = -0.5 * expm1(-G);
    if (0.5 - m < 1e-6) return -1.0;
    double y = (m < 0.3) ? log(m / fmax(log(1.0 / m) - 1.0, 1.0)) : log(1.0 / (6.0 * (0.5 - m)));
    for (int it = 0; it < 200; it++) {
        double A = exp(y);
        double f = wentzel_mean(A) - m;
        double dm = (A > 100.0) ? (1.0 / (6.0 * A * A) - 1.0 / (6.0 * A * A * A)) : ((1.0 + 2.0 * A) * log1p(1.0 / A) - 2.0);
        double step = f / (A * dm);
        if (step > 2.0) step = 2.0;
        if (step < -2.0) step = -2.0;
        y -= step;
        if (fabs(step) < 1e-13) break;
    }
    return exp(y);
}

static double sample_ms_mu(double A, double xi) {
    if (A < 0.0) return xi;            /* isotropic */
    return A * xi / (1.0 - xi + A);
}

/* Rotate unit direction u by polar cos ct and azimuth phi. */
static void rotate(double u[3], double ct, double phi) {
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double cp = cos(phi), sp = sin(phi);
    double w = u[2];
    if (fabs(w) > 0.99999) {          /* polar frame near the z axis */
        double sg = (w > 0) ? 1.0 : -1.0;
        u[0] = st * cp; u[1] = st * sp; u[2] = sg * ct;
    } else {
        double tmp = sqrt(1.0 - w * w);
        double nu = u[0] * ct + st * (u[0] * w * cp - u[1] * sp) / tmp;
        double nv = u[1] * ct + st * (u[1] * w * cp + u[0] * sp) / tmp;
        double nw = w * ct - tmp * st * cp;
        u[0] = nu; u[1] = nv; u[2] = nw;
    }
    double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    u[0] /= n; u[1] /= n; u[2] /= n;
}

/* ------------------------------------------------------------------------ */
/* Problem description and results (mirrored by the Python wrapper).         */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int16_t* hu; int nx, ny, nz; double vox[3]; double origin[3];
    int n_layers; int layer_mat[O_MAXL]; double layer_thick[O_MAXL]; double layer_rho[O_MAXL];
    int sens_layer; int npx, npy; double pitch;
    int n_seg, n_pairs; const double* pair_edges; const double* leaves; const double* jaws; const double* mu;
    double gantry_deg, sad, sid; double iso[3];
    int coupled; double e_max, mono_e, pcut, ecut, wcc, wcb, step_frac; int n_batches; int max_steps;
    double leaf_trans;           /* fluence fraction through closed leaves (0: ideal MLC) */
    double jaw_trans;            /* fluence fraction through the jaws (0: opaque) */
    double tg_width;             /* tongue-and-groove strip width at the isocentre plane, cm */
    double leaf_gap;             /* dosimetric leaf gap of an open pair, cm */
    double leaf_thick;           /* tungsten leaf slab thickness along the beam, cm (0: no leaf slab) */
    double jaw_thick;            /* tungsten jaw slab thickness along the beam, cm (0: no jaw slab) */
} orc_problem;

enum { C_FLIGHTS_CT, C_REAL_CT, C_COMPTON, C_PHOTO, C_PAIR, C_ESTEP_CT, C_ESTEP_EPID, C_MOLLER, C_BREM,
       C_PRIM_EPID, C_UNCOLLIDED, C_LOST, C_FLIGHTS_EPID, C_ELECTRONS, C_POSITRONS, C_PHOTONS2, C_NCOUNT };

typedef struct {
    double* tally;               /* [B][npy][npx] MeV */
    double e_src, e_ct, e_epid[O_MAXL], e_esc, e_lost;
    uint64_t counters[C_NCOUNT];
    double* vox;                 /* [nz][ny][nx] MeV deposited per CT voxel, or NULL (patient dose off) */
} orc_result;

/* ------------------------------------------------------------------------ */
/* Transport.                                                                 */
/* ------------------------------------------------------------------------ */
enum { Z_CT = 0, Z_EPID = 1 };
enum { P_PHOTON = 0, P_ELECTRON = 1, P_POSITRON = 2 };

typedef struct {
    int type, zone;
    double x[3], u[3], E;
    int cell[3];                 /* CT voxel index, or [0] = EPID layer */
    int collided;                /* primaries only: has had a real interaction */
    double tau;                  /* charged particles: optical depth left to the next tentative hard event
                                    against the step majorants; <= 0: none drawn yet */
    int prim;                    /* the probe's primary particle (test hook only; children are 0) */
    o_rng rng;
} o_part;

/* ------------------------------------------------------------------------ */
/* Test probe (orc_pencil only): facts about one primary particle per history */
/* and kinematic checks of each interaction, gathered for the CPU pins.  The  */
/* transport below only reads `no_ms` / `no_hard` from it and otherwise       */
/* records; with no probe (every orc_run) nothing changes.                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    /* inputs */
    int type;                    /* primary: 0 photon, 1 electron, 2 positron */
    double E;                    /* its kinetic energy, MeV */
    double x[3], u[3];           /* start and direction, patient frame (a charged primary starts inside the CT) */
    int no_ms, no_hard;          /* switches: no multiple-scattering deflection; no hard events */
    int macro_M;                 /* macro-cell size override for the Woodcock majorant (0: default rule) */
    int64_t cap;                 /* capacity of the sample arrays below */
    /* per-history outputs (arrays of n, each may be NULL) */
    double* path;                /* track length of a charged primary, cm */
    double* hard_T;              /* primary's kinetic energy when its first hard event happens, or -1 */
    int32_t* hard_type;          /* that event: 0 Moller, 1 bremsstrahlung, -1 none */
    int32_t* first_layer;        /* primary photon's first real interaction: EPID layer, -1 CT, -2 none */
    double* first_pos;           /* [n][3] its point, beam frame (EPID interactions only) */
    double* end_pos;             /* [n][3] where a charged primary stops (patient frame), NaN if it never stops */
    int64_t* first_pixel;        /* sensitive-layer pixel y*npx+x that its first deposit went to, or -1 */
    /* samples (first `cap` events of each kind) */
    double* pair_frac;           /* T- / (E - 2 mc^2) of each pair event */
    double* annih_cos;           /* cos(polar angle) of the first photon of each annihilation */
    double* annih_phi;           /* its azimuth, [0, 2 pi) */
    double* brem_x;              /* ln(k / wcb) / ln(T / wcb) of each hard bremsstrahlung photon */
    double* compton_phi;         /* azimuth of the scattered photon about the incident direction */
    /* aggregate outputs */
    uint64_t n_exit_uncollided;  /* primary photons leaving the EPID's far face with no real interaction */
    uint64_t n_compton, n_moller, n_brem, n_pair, n_annih, n_pos_escape, n_pos_born;
    double compton_dev;          /* max over Compton events with |w0| <= 0.99999 (the general rotation frame):
                                    | |E0 u0 - E1 u1| - p_e | / E0 and |u0.u1 - cos| */
    double polar_dev;            /* the Compton and Moller figures for events in the polar frame
                                    (|w0| > 0.99999), which takes u0 as the z axis itself */
    double moller_dev;           /* max | p0 u0 - pW uW - pT uT | / p0 (general frame; polar frame: polar_dev) */
    double brem_dev;             /* max | photon direction - electron direction | */
    double pair_dev;             /* max | T- + T+ - (E - 2 mc^2) | */
    double annih_dev;            /* max |u1 + u2|, |E1 - mc^2|, |E2 - mc^2| */
    double unit_dev;             /* max | |u| - 1 | of any direction set by an interaction */
    /* working state */
    int64_t hidx;                /* index of the current history in the per-history arrays */
    int first_done, pix_done, hard_done;
} orc_probe;

typedef struct {
    const orc_problem* P;
    double ex[3], ey[3], ez[3];       /* beam-frame axes in patient coordinates */
    double zplane[O_MAXL + 1];        /* EPID layer planes, beam-frame Z, top first */
    double half_w[2];                 /* EPID lateral half widths */
    double rho_max[4];                /* per CT material */
    int mat_present[4];
    int mgM, mg[3];                   /* macro-cells: M voxels per side, count per axis */
    double* mg_low;                   /* per macro-cell max density of air, lung, water voxels */
    double* mg_bone;                  /* per macro-cell max density of bone voxels */
    unsigned char* hom;               /* per voxel: 1 if homogeneous (see ctx_homogeneity) */
    double* rect;                     /* source rectangles: x0,x1,y0,y1 */
    int* rflag;                       /* per rectangle: bit 0 behind a closed leaf, bit 1 outside the jaws */
    double* cdf;                      /* cumulative weight */
    int n_rect;
    /* per worker */
    double* tally; double e_src, e_ct, e_epid[O_MAXL], e_esc, e_lost;
    double* vox;                      /* this worker's voxel tally (patient dose), or NULL */
    uint64_t cnt[C_NCOUNT];
    uint64_t hist;
    o_part* stack; int sp, cap;
    orc_probe* probe;                 /* test hook, NULL in every orc_run */
} o_ctx;

/* HU -> density (g/cm^3) and material (stated reading of the curve in Sec. 2.1.2). */
void orc_hu_to_rho_mat(int hu, double* rho, int* mat) {
    if (hu < -1024) hu = -1024;
    if (hu > 3071) hu = 3071;
    double r = (hu <= 0) ? 1.0 + hu / 1000.0 : 1.0 + 0.6 * hu / 1000.0;
    if (r < 0.001205) r = 0.001205;
    *rho = r;
    *mat = (hu < -900) ? 0 : (hu < -200) ? 1 : (hu < 300) ? 2 : 3;
}

static void to_patient(const o_ctx* c, const double b[3], double p[3]) {
    for (int i = 0; i < 3; i++) p[i] = c->P->iso[i] + b[0] * c->ex[i] + b[1] * c->ey[i] + b[2] * c->ez[i];
}
static void to_patient_dir(const o_ctx* c, const double b[3], double p[3]) {
    for (int i = 0; i < 3; i++) p[i] = b[0] * c->ex[i] + b[1] * c->ey[i] + b[2] * c->ez[i];
}
static void to_beam(const o_ctx* c, const double p[3], double b[3]) {
    double d[3] = {p[0] - c->P->iso[0], p[1] - c->P->iso[1], p[2] - c->P->iso[2]};
    b[0] = d[0] * c->ex[0] + d[1] * c->ex[1] + d[2] * c->ex[2];
    b[1] = d[0] * c->ey[0] + d[1] * c->ey[1] + d[2] * c->ey[2];
    b[2] = d[0] * c->ez[0] + d[1] * c->ez[1] + d[2] * c->ez[2];
}
static void to_beam_dir(const o_ctx* c, const double p[3], double b[3]) {
    b[0] = p[0] * c->ex[0] + p[1] * c->ex[1] + p[2] * c->ex[2];
    b[1] = p[0] * c->ey[0] + p[1] * c->ey[1] + p[2] * c->ey[2];
    b[2] = p[0] * c->ez[0] + p[1] * c->ez[1] + p[2] * c->ez[2];
}

static void push(o_ctx* c, const o_part* p) {
    if (c->sp == c->cap) {
        c->cap = c->cap ? 2 * c->cap : 64;
        c->stack = (o_part*)realloc(c->stack, sizeof(o_part) * c->cap);
    }
    c->stack[c->sp++] = *p;
}

static double rest_extra(const o_part* p) { return (p->type == P_POSITRON) ? 2.0 * O_MC2 : 0.0; }

/* The probe's first-deposit record: the sensitive-layer pixel, or -1. */
static void probe_first_deposit(o_ctx* c, const o_part* p, int64_t pixel) {
    orc_probe* Q = c->probe;
    if (!Q || !p->prim || Q->pix_done) return;
    Q->pix_done = 1;
    if (Q->first_pixel) Q->first_pixel[Q->hidx] = pixel;
}

static void deposit(o_ctx* c, const o_part* p, const double pos[3], int layer, double dE) {
    if (dE == 0.0) return;
    if (p->zone == Z_CT) {
        c->e_ct += dE;
        /* patient dose: the energy goes to the voxel the particle is in */
        if (c->vox) c->vox[((size_t)p->cell[2] * c->P->ny + p->cell[1]) * c->P->nx + p->cell[0]] += dE;
        probe_first_deposit(c, p, -1);
        return;
    }
    c->e_epid[layer] += dE;
    const orc_problem* P = c->P;
    if (layer != P->sens_layer) { probe_first_deposit(c, p, -1); return; }
    int ix = (int)floor((pos[0] + c->half_w[0]) / P->pitch);
    int iy = (int)floor((pos[1] + c->half_w[1]) / P->pitch);
    if (ix < 0) ix = 0;
    if (ix >= P->npx) ix = P->npx - 1;
    if (iy < 0) iy = 0;
    if (iy >= P->npy) iy = P->npy - 1;
    probe_first_deposit(c, p, (int64_t)iy * P->npx + ix);
    int b = (int)(c->hist % (uint64_t)P->n_batches);
    c->tally[((size_t)b * P->npy + iy) * P->npx + ix] += dE;
}

/* Energy leaving the world (escape), with the probe's count of positrons
 * that end this way instead of annihilating. */
static void escape(o_ctx* c, const o_part* p, double E) {
    c->e_esc += E;
    if (c->probe && p->type == P_POSITRON) c->probe->n_pos_escape++;
}

static void probe_max(double* acc, double v) { if (v > *acc) *acc = v; }

/* The probe's record of where a charged primary comes to rest. */
static void probe_end(o_ctx* c, const o_part* p, const double pos[3]) {
    orc_probe* Q = c->probe;
    if (!Q || !p->prim || !Q->end_pos) return;
    for (int a = 0; a < 3; a++) Q->end_pos[3 * Q->hidx + a] = pos[a];
}

static void probe_unit(o_ctx* c, const double u[3]) {
    probe_max(&c->probe->unit_dev, fabs(sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) - 1.0));
}

/* Azimuth of direction v about axis a in a frame fixed by a alone. */
static double azimuth_about(const double a[3], const double v[3]) {
    double r[3] = {1.0, 0.0, 0.0};
    if (fabs(a[0]) > 0.6) { r[0] = 0.0; r[1] = 1.0; }
    double e1[3] = {a[1] * r[2] - a[2] * r[1], a[2] * r[0] - a[0] * r[2], a[0] * r[1] - a[1] * r[0]};
    double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; i++) e1[i] /= n1;
    double e2[3] = {a[1] * e1[2] - a[2] * e1[1], a[2] * e1[0] - a[0] * e1[2], a[0] * e1[1] - a[1] * e1[0]};
    double ph = atan2(v[0] * e2[0] + v[1] * e2[1] + v[2] * e2[2], v[0] * e1[0] + v[1] * e1[1] + v[2] * e1[2]);
    return ph < 0.0 ? ph + 2.0 * O_PI : ph;
}

/* Momentum |p| of an electron of kinetic energy T, MeV/c. */
static double p_of_T(double T) { return sqrt(T * (T + 2.0 * O_MC2)); }

static void ct_props(const o_ctx* c, const int idx[3], double* rho, int* mat) {
    const orc_problem* P = c->P;
    int hu = P->hu[((size_t)idx[2] * P->ny + idx[1]) * P->nx + idx[0]];
    orc_hu_to_rho_mat(hu, rho, mat);
}

/* Send a particle that has left the CT (or never entered it) across the
 * vacuum gap: into the EPID's top layer if its line meets the detector face,
 * otherwise out of the world. */
static void transfer_to_epid(o_ctx* c, o_part* p) {
    double b[3], ub[3];
    to_beam(c, p->x, b);
    to_beam_dir(c, p->u, ub);
    double Eexit = p->E + rest_extra(p);
    if (ub[2] >= 0.0) { escape(c, p, Eexit); return; }
    /* Any point of the vacuum line will do: a Woodcock flight may have carried
     * the photon past the detector plane, but the CT lies wholly above it, so
     * the line's crossing of the detector face is always downstream of the
     * true exit point. */
    double t = (c->zplane[0] - b[2]) / ub[2];
    double X = b[0] + t * ub[0], Y = b[1] + t * ub[1];
    if (!(fabs(X) < c->half_w[0] && fabs(Y) < c->half_w[1])) { escape(c, p, Eexit); return; }
    p->zone = Z_EPID;
    p->x[0] = X; p->x[1] = Y; p->x[2] = c->zplane[0];
    p->u[0] = ub[0]; p->u[1] = ub[1]; p->u[2] = ub[2];
    p->cell[0] = 0;
    if (p->type == P_PHOTON && p->rng.ord == 0 && !p->collided) c->cnt[C_UNCOLLIDED]++;
    if (p->type == P_PHOTON && p->rng.ord == 0) c->cnt[C_PRIM_EPID]++;
    push(c, p);
}

static void enter_world(o_ctx* c, o_part* p) {
    /* p is a photon at the source, patient frame.  Move it to the CT box entry
     * if its line meets the box, else send it to the EPID. */
    const orc_problem* P = c->P;
    double lo[3], hi[3];
    int n[3] = {P->nx, P->ny, P->nz};
    double t0 = -INFINITY, t1 = INFINITY;
    for (int a = 0; a < 3; a++) {
        lo[a] = P->origin[a];
        hi[a] = P->origin[a] + n[a] * P->vox[a];
        if (p->u[a] != 0.0) {
            double ta = (lo[a] - p->x[a]) / p->u[a], tb = (hi[a] - p->x[a]) / p->u[a];
            if (ta > tb) { double t = ta; ta = tb; tb = t; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        } else if (p->x[a] < lo[a] || p->x[a] > hi[a]) {
            t0 = INFINITY;
        }
    }
    if (t0 < t1 && t1 > 0.0) {
        double t = fmax(t0, 0.0);
        for (int a = 0; a < 3; a++) p->x[a] += t * p->u[a];
        p->zone = Z_CT;
        push(c, p);
    } else {
        transfer_to_epid(c, p);
    }
}

static void make_child(const o_part* parent, o_part* ch, int type, uint32_t slot) {
    memset(ch, 0, sizeof(*ch));
    ch->type = type;
    ch->zone = parent->zone;
    ch->cell[0] = parent->cell[0]; ch->cell[1] = parent->cell[1]; ch->cell[2] = parent->cell[2];
    ch->x[0] = parent->x[0]; ch->x[1] = parent->x[1]; ch->x[2] = parent->x[2];
    ch->collided = 1;
    ch->rng = parent->rng;
    ch->rng.ord = orc_child_ordinal(parent->rng.ord, parent->rng.d, slot);
    ch->rng.d = 0;
    ch->rng.cvalid = 0;
}

/* Annihilation at rest: two mc^2 photons, isotropic, back to back; they are
 * the parent's children with slots 0 and 1 after its two direction draws. */
static void annihilate(o_ctx* c, o_part* parent) {
    double ct = 2.0 * rng_u(&parent->rng) - 1.0;
    double ph = 2.0 * O_PI * rng_u(&parent->rng);
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double d[3] = {st * cos(ph), st * sin(ph), ct};
    double gu[2][3], gE[2];
    for (int k = 0; k < 2; k++) {
        o_part g;
        make_child(parent, &g, P_PHOTON, (uint32_t)k);
        double sg = k ? -1.0 : 1.0;
        g.u[0] = sg * d[0]; g.u[1] = sg * d[1]; g.u[2] = sg * d[2];
        g.E = O_MC2;
        for (int a = 0; a < 3; a++) gu[k][a] = g.u[a];
        gE[k] = g.E;
        c->cnt[C_PHOTONS2]++;
        push(c, &g);
    }
    orc_probe* Q = c->probe;
    if (Q) {
        double sum = sqrt((gu[0][0] + gu[1][0]) * (gu[0][0] + gu[1][0]) + (gu[0][1] + gu[1][1]) * (gu[0][1] + gu[1][1]) +
                          (gu[0][2] + gu[1][2]) * (gu[0][2] + gu[1][2]));
        probe_max(&Q->annih_dev, fmax(sum, fmax(fabs(gE[0] - O_MC2), fabs(gE[1] - O_MC2))));
        probe_unit(c, gu[0]);
        if ((int64_t)Q->n_annih < Q->cap) {
            if (Q->annih_cos) Q->annih_cos[Q->n_annih] = gu[0][2];
            if (Q->annih_phi) { double a = atan2(gu[0][1], gu[0][0]); Q->annih_phi[Q->n_annih] = a < 0 ? a + 2.0 * O_PI : a; }
        }
        Q->n_annih++;
    }
}

static int layer_mat(const o_ctx* c, int l) { return c->P->layer_mat[l]; }

/* The probe's record of the primary photon's first real interaction: the
 * EPID layer (or -1 in the CT) and, in the EPID, the beam-frame point. */
static void probe_first_interaction(o_ctx* c, const o_part* p, int layer) {
    orc_probe* Q = c->probe;
    if (!Q || !p->prim || Q->first_done) return;
    Q->first_done = 1;
    if (Q->first_layer) Q->first_layer[Q->hidx] = layer;
    if (Q->first_pos && layer >= 0)
        for (int a = 0; a < 3; a++) Q->first_pos[3 * Q->hidx + a] = p->x[a];
}

/* Emit an electron or positron of kinetic energy T created by `parent`, or
 * deposit it when transport is off or T is at the cutoff. */
static void emit_charged(o_ctx* c, o_part* parent, int type, double T, const double dir[3], uint32_t slot,
                         int layer) {
    const orc_problem* P = c->P;
    if (P->coupled && T > P->ecut + O_TSTOP) {
        o_part e;
        make_child(parent, &e, type, slot);
        e.u[0] = dir[0]; e.u[1] = dir[1]; e.u[2] = dir[2];
        e.E = T;
        c->cnt[type == P_POSITRON ? C_POSITRONS : C_ELECTRONS]++;
        push(c, &e);
    } else {
        deposit(c, parent, parent->x, layer, T);
    }
}

/* A real photon interaction at p->x in material m.  Returns 1 if the photon
 * survives (Compton above the cutoff), 0 if it is absorbed. */
static int photon_interact(o_ctx* c, o_part* p, int m, int layer) {
    const orc_problem* P = c->P;
    double mu[3];
    orc_mu_photon(m, p->E, mu);
    double tot = mu[0] + mu[1] + mu[2];
    double xi = rng_u(&p->rng);
    p->collided = 1;
    if (xi * tot < mu[0]) {
        c->cnt[C_COMPTON]++;
        double eps, ct;
        sample_kn(&p->rng, p->E, &eps, &ct);
        double phi = 2.0 * O_PI * rng_u(&p->rng);
        double E0 = p->E, E1 = eps * E0;
        double u0[3] = {p->u[0], p->u[1], p->u[2]};
        rotate(p->u, ct, phi);
        double T = E0 - E1;
        double pe[3] = {E0 * u0[0] - E1 * p->u[0], E0 * u0[1] - E1 * p->u[1], E0 * u0[2] - E1 * p->u[2]};
        double n = sqrt(pe[0] * pe[0] + pe[1] * pe[1] + pe[2] * pe[2]);
        orc_probe* Q = c->probe;
        if (Q) {
            /* momentum balance with the electron's |p| from its kinetic energy, and the scattering angle */
            double* dev = (fabs(u0[2]) > 0.99999) ? &Q->polar_dev : &Q->compton_dev;
            probe_max(dev, fabs(n - p_of_T(T)) / E0);
            probe_max(dev, fabs(u0[0] * p->u[0] + u0[1] * p->u[1] + u0[2] * p->u[2] - ct));
            probe_unit(c, p->u);
            if ((int64_t)Q->n_compton < Q->cap && Q->compton_phi) Q->compton_phi[Q->n_compton] = azimuth_about(u0, p->u);
            Q->n_compton++;
        }
        if (n > 0.0) { pe[0] /= n; pe[1] /= n; pe[2] /= n; } else { pe[0] = u0[0]; pe[1] = u0[1]; pe[2] = u0[2]; }
        emit_charged(c, p, P_ELECTRON, T, pe, 0, layer);
        p->E = E1;
        if (p->E < P->pcut) { deposit(c, p, p->x, layer, p->E); return 0; }
        return 1;
    } else if (xi * tot < mu[0] + mu[1]) {
        c->cnt[C_PHOTO]++;
        emit_charged(c, p, P_ELECTRON, p->E, p->u, 0, layer);
        return 0;
    } else {
        c->cnt[C_PAIR]++;
        double avail = p->E - 2.0 * O_MC2;
        double xu = rng_u(&p->rng);
        double Tm = xu * avail, Tp = avail - Tm;
        orc_probe* Q = c->probe;
        if (Q) {
            probe_max(&Q->pair_dev, fabs(Tm + Tp - (p->E - 2.0 * O_MC2)));
            if ((int64_t)Q->n_pair < Q->cap && Q->pair_frac) Q->pair_frac[Q->n_pair] = Tm / avail;
            Q->n_pair++;
            Q->n_pos_born++;
        }
        if (P->coupled) {
            emit_charged(c, p, P_ELECTRON, Tm, p->u, 0, layer);
            if (Tp > P->ecut + O_TSTOP) {
                emit_charged(c, p, P_POSITRON, Tp, p->u, 1, layer);
            } else {
                /* a positron born at the cutoff stops and annihilates at once */
                deposit(c, p, p->x, layer, Tp);
                annihilate(c, p);
            }
        } else {
            deposit(c, p, p->x, layer, Tm + Tp);
            annihilate(c, p);
        }
        return 0;
    }
}

/* Largest per-gram attenuation of the non-bone CT materials and of bone. */
static void mu_groups(double E, double* mu_low, double* mu_bone) {
    *mu_low = fmax(mu_total(0, E), fmax(mu_total(1, E), mu_total(2, E)));
    *mu_bone = mu_total(3, E);
}

/* One Woodcock flight with a piecewise-constant majorant: an optical depth
 * tau = -ln(xi) is spent along the ray across macro-cells, each with majorant
 * Sigma_c = max(rho_low,c mu_low(E), rho_bone,c mu_bone(E)).  Returns 1 with
 * the tentative collision's voxel (kept inside its macro-cell) and Sigma_c, or
 * 0 when the ray leaves the CT (x is then on the box's face). */
static int ct_flight(const o_ctx* c, double x[3], const double u[3], double E, o_rng* r, int idx[3], double* Sc_out) {
    const orc_problem* P = c->P;
    const int n[3] = {P->nx, P->ny, P->nz};
    const int M = c->mgM;
    double mul, mub;
    mu_groups(E, &mul, &mub);
    rng_align(r);
    double tau = -log(rng_u(r));
    int cm[3];
    for (int a = 0; a < 3; a++) {
        int k = (int)floor((x[a] - P->origin[a]) / (M * P->vox[a]));
        cm[a] = k < 0 ? 0 : (k >= c->mg[a] ? c->mg[a] - 1 : k);
    }
    for (;;) {
        size_t cc = ((size_t)cm[2] * c->mg[1] + cm[1]) * c->mg[0] + cm[0];
        double Sc = fmax(c->mg_low[cc] * mul, c->mg_bone[cc] * mub);
        double d = INFINITY;
        int ax = 0;
        for (int a = 0; a < 3; a++) {
            double da = INFINITY;
            if (u[a] > 0.0) {
                int hi = (cm[a] + 1) * M < n[a] ? (cm[a] + 1) * M : n[a];
                da = (P->origin[a] + hi * P->vox[a] - x[a]) / u[a];
            } else if (u[a] < 0.0) {
                da = (P->origin[a] + cm[a] * M * P->vox[a] - x[a]) / u[a];
            }
            if (da < d) { d = da; ax = a; }
        }
        if (d < 0.0) d = 0.0;
        if (tau < Sc * d) {
            double s = tau / Sc;
            for (int a = 0; a < 3; a++) x[a] += s * u[a];
            for (int a = 0; a < 3; a++) {
                int k = (int)floor((x[a] - P->origin[a]) / P->vox[a]);
                int lo = cm[a] * M, hi = ((cm[a] + 1) * M < n[a] ? (cm[a] + 1) * M : n[a]) - 1;
                idx[a] = k < lo ? lo : (k > hi ? hi : k);
            }
            *Sc_out = Sc;
            return 1;
        }
        tau -= Sc * d;
        for (int a = 0; a < 3; a++) x[a] += d * u[a];
        cm[ax] += (u[ax] > 0.0) ? 1 : -1;
        if (cm[ax] < 0 || cm[ax] >= c->mg[ax]) return 0;
    }
}

/* Photon transport in the CT: flights until a tentative collision is real
 * (probability Sigma_voxel / Sigma_c) or the photon leaves the CT. */
static void photon_ct(o_ctx* c, o_part* p) {
    const orc_problem* P = c->P;
    for (int f = 0; f < P->max_steps; f++) {
        int idx[3];
        double Sc;
        c->cnt[C_FLIGHTS_CT]++;
        if (!ct_flight(c, p->x, p->u, p->E, &p->rng, idx, &Sc)) { transfer_to_epid(c, p); return; }
        double rho; int m;
        ct_props(c, idx, &rho, &m);
        double sig = rho * mu_total(m, p->E);
        if (!(rng_u(&p->rng) * Sc < sig)) continue;      /* virtual */
        c->cnt[C_REAL_CT]++;
        p->cell[0] = idx[0]; p->cell[1] = idx[1]; p->cell[2] = idx[2];
        probe_first_interaction(c, p, -1);
        if (!photon_interact(c, p, m, 0)) return;
    }
    c->e_lost += p->E;
    c->cnt[C_LOST]++;
}

/* distance along u to leave EPID layer l: which = 0 (z plane), 1 (x edge), 2 (y edge) */
static double epid_dist(const o_ctx* c, const double x[3], const double u[3], int l, int* which) {
    double dz = INFINITY, dx = INFINITY, dy = INFINITY;
    if (u[2] < 0.0) dz = (c->zplane[l + 1] - x[2]) / u[2];
    else if (u[2] > 0.0) dz = (c->zplane[l] - x[2]) / u[2];
    if (u[0] > 0.0) dx = (c->half_w[0] - x[0]) / u[0];
    else if (u[0] < 0.0) dx = (-c->half_w[0] - x[0]) / u[0];
    if (u[1] > 0.0) dy = (c->half_w[1] - x[1]) / u[1];
    else if (u[1] < 0.0) dy = (-c->half_w[1] - x[1]) / u[1];
    double d = dz; *which = 0;
    if (dx < d) { d = dx; *which = 1; }
    if (dy < d) { d = dy; *which = 2; }
    return fmax(d, 0.0);
}

static void photon_epid(o_ctx* c, o_part* p) {
    const orc_problem* P = c->P;
    for (int f = 0; f < P->max_steps; f++) {
        rng_align(&p->rng);
        double tau = -log(rng_u(&p->rng));
        c->cnt[C_FLIGHTS_EPID]++;
        for (;;) {
            int l = p->cell[0];
            double mu = P->layer_rho[l] * mu_total(layer_mat(c, l), p->E);
            int which;
            double d = epid_dist(c, p->x, p->u, l, &which);
            if (tau < mu * d) {
                double s = tau / mu;
                for (int a = 0; a < 3; a++) p->x[a] += s * p->u[a];
                break;
            }
            tau -= mu * d;
            for (int a = 0; a < 3; a++) p->x[a] += d * p->u[a];
            if (which != 0) { escape(c, p, p->E); return; }
            int nl = l + (p->u[2] < 0.0 ? 1 : -1);
            if (nl < 0 || nl >= P->n_layers) {
                if (c->probe && p->prim && !p->collided && nl >= P->n_layers) c->probe->n_exit_uncollided++;
                escape(c, p, p->E);
                return;
            }
            p->cell[0] = nl;
        }
        probe_first_interaction(c, p, p->cell[0]);
        if (!photon_interact(c, p, layer_mat(c, p->cell[0]), p->cell[0])) return;
    }
    c->e_lost += p->E;
    c->cnt[C_LOST]++;
}

/* CT voxel boundary distance for charged-particle steps. */
static double ct_dist(const o_ctx* c, const double x[3], const double u[3], const int cell[3], int* axis) {
    const orc_problem* P = c->P;
    double best = INFINITY; *axis = -1;
    for (int a = 0; a < 3; a++) {
        double d = INFINITY;
        if (u[a] > 0.0) d = (P->origin[a] + (cell[a] + 1) * P->vox[a] - x[a]) / u[a];
        else if (u[a] < 0.0) d = (P->origin[a] + cell[a] * P->vox[a] - x[a]) / u[a];
        if (d < best) { best = d; *axis = a; }
    }
    return fmax(best, 0.0);
}

/* Where the second segment of a CT hinge step may run through faces: from x
 * along u for length len, starting in voxel cell, it ends in voxel end (by
 * floor of the end point).  It runs through if cell is homogeneous (c->hom)
 * and end lies within O_HOM_R voxels of it along every axis. */
static int leg_through(const o_ctx* c, const double x[3], const double u[3], const int cell[3], double len,
                       int end[3]) {
    const orc_problem* P = c->P;
    if (!c->hom[((size_t)cell[2] * P->ny + cell[1]) * P->nx + cell[0]]) return 0;
    for (int a = 0; a < 3; a++) {
        end[a] = (int)floor((x[a] + len * u[a] - P->origin[a]) / P->vox[a]);
        if (abs(end[a] - cell[a]) > O_HOM_R) return 0;
    }
    return 1;
}

/* Walk a straight segment of length len from x along u, starting in voxel
 * cell, face by face (crossing at most O_MAXFACES faces): the voxels it
 * passes (cells[k]) and the length in each (lens[k]), in order; returns
 * their number. */
#define O_MAXFACES (3 * O_HOM_R)
static int leg_walk(const o_ctx* c, const double x[3], const double u[3], const int cell[3], double len,
                    int cells[][3], double* lens) {
    double q[3] = {x[0], x[1], x[2]};
    int cc[3] = {cell[0], cell[1], cell[2]};
    double left = len;
    for (int k = 0; k <= O_MAXFACES; k++) {
        int ax;
        double d = ct_dist(c, q, u, cc, &ax);
        cells[k][0] = cc[0]; cells[k][1] = cc[1]; cells[k][2] = cc[2];
        if (d >= left || k == O_MAXFACES) { lens[k] = left; return k + 1; }
        lens[k] = d;
        left -= d;
        for (int a = 0; a < 3; a++) q[a] += d * u[a];
        cc[ax] += (u[ax] > 0.0) ? 1 : -1;
    }
    return 0;
}

static void electron(o_ctx* c, o_part* p) {
    const orc_problem* P = c->P;
    const double tcut = P->ecut, tstop = P->ecut + O_TSTOP;
    for (int step = 0; step < P->max_steps; step++) {
        double rho; int m; int layer = 0;
        if (p->zone == Z_CT) {
            ct_props(c, p->cell, &rho, &m);
            c->cnt[C_ESTEP_CT]++;
        } else {
            layer = p->cell[0];
            rho = P->layer_rho[layer];
            m = layer_mat(c, layer);
            c->cnt[C_ESTEP_EPID]++;
        }
        double T = p->E;
        rng_align(&p->rng);
        /* (a) energy-loss limited step with midpoint stopping power */
        double dEt = P->step_frac * T;
        if (T - dEt < tstop) dEt = T - tcut;
        double Tm = T - 0.5 * dEt;
        double L = rho * (orc_lcol(m, Tm, P->wcc) + orc_lrad_soft(m, Tm, P->wcb));
        double sE = dEt / L;
        /* (b) distance to the next tentative hard event: an optical depth
         * tau = -ln(xi), taken when none is pending, is spent along the path
         * against each step's majorant Sh (the hard cross section at the
         * step's start energy, which bounds it over the step because it never
         * decreases with T), across steps and faces, until it runs out */
        double Sh = (c->probe && c->probe->no_hard) ? 0.0
                    : rho * (orc_sigma_moller(m, T, P->wcc) + orc_sigma_brem(m, T, P->wcb));
        const double xt = rng_u(&p->rng);            /* drawn every step, used when no depth is pending */
        if (!(p->tau > 0.0)) p->tau = -log(xt);
        double sh = p->tau / Sh;
        /* (c) distance to the cell boundary */
        int ax;
        double sb = (p->zone == Z_CT) ? ct_dist(c, p->x, p->u, p->cell, &ax) : epid_dist(c, p->x, p->u, layer, &ax);
        double s = sE; int lim = 0;
        if (sh < s) { s = sh; lim = 1; }
        double xh = rng_u(&p->rng), xmu = rng_u(&p->rng), xph = rng_u(&p->rng);
        /* Face rule.  In the CT the hinge is placed on the planned step s, which
         * ignores voxel faces: a step whose hinge lies beyond the face becomes a
         * face step (straight to the face).  In the EPID, whose layers are
         * different materials, every step that would reach a layer face is a
         * face step. */
        if ((p->zone == Z_CT) ? (xh * s >= sb) : (sb < s)) { s = sb; lim = 2; }
        /* multiple-scattering deflection for the distance s, with the scattering
         * power at the mid-step energy */
        double G = s * rho * orc_lambda1_inv(m, T - 0.5 * dEt * (s / sE));
        double A = orc_wentzel_A(G);
        double mu = (G > 0.0 && !(c->probe && c->probe->no_ms)) ? sample_ms_mu(A, xmu) : 0.0;
        const int track = c->probe && p->prim && c->probe->path;
        if (lim == 2) {
            /* Face step: straight to the face, energy deposited at the segment
             * midpoint, the face crossed, then the deflection for the distance
             * travelled applied.  (A hinge inside such a step would leave the
             * particle just short of the face after a small deflection, and the
             * next, ever-shorter steps would end where rounding decides the
             * crossing.) */
            double mid[3], hc[3] = {p->cell[0], p->cell[1], p->cell[2]};
            for (int a = 0; a < 3; a++) { mid[a] = p->x[a] + 0.5 * s * p->u[a]; p->x[a] += s * p->u[a]; }
            if (track) c->probe->path[c->probe->hidx] += s;
            double dE = dEt * (s / sE);
            double Tn = T - dE;
            p->tau -= s * Sh;
            o_part here = *p;
            if (Tn <= tstop) {
                probe_end(c, p, mid);
                deposit(c, &here, mid, (int)hc[0], dE + Tn);
                if (p->type == P_POSITRON) {
                    p->x[0] = mid[0]; p->x[1] = mid[1]; p->x[2] = mid[2];
                    annihilate(c, p);
                }
                return;
            }
            deposit(c, &here, mid, (int)hc[0], dE);
            p->E = Tn;
            if (p->zone == Z_CT) {
                p->cell[ax] += (p->u[ax] > 0.0) ? 1 : -1;
                int n[3] = {P->nx, P->ny, P->nz};
                if (p->cell[ax] < 0 || p->cell[ax] >= n[ax]) { transfer_to_epid(c, p); return; }
            } else {
                if (ax != 0) { escape(c, p, p->E + rest_extra(p)); return; }
                int nl = layer + (p->u[2] < 0.0 ? 1 : -1);
                if (nl < 0 || nl >= P->n_layers) { escape(c, p, p->E + rest_extra(p)); return; }
                p->cell[0] = nl;
            }
            rotate(p->u, 1.0 - 2.0 * mu, 2.0 * O_PI * xph);
            continue;
        }
        /* random hinge: first segment, deflection, second segment */
        double s1 = xh * s;
        for (int a = 0; a < 3; a++) p->x[a] += s1 * p->u[a];
        double hinge[3] = {p->x[0], p->x[1], p->x[2]};
        int hcell[3] = {p->cell[0], p->cell[1], p->cell[2]};
        rotate(p->u, 1.0 - 2.0 * mu, 2.0 * O_PI * xph);
        double s2 = s - s1;
        int ax2;
        double sb2 = (p->zone == Z_CT) ? ct_dist(c, p->x, p->u, p->cell, &ax2) : epid_dist(c, p->x, p->u, layer, &ax2);
        int crossed = 0, through = 0, ecell[3];
        if (s2 >= sb2) {
            /* In the CT the second segment runs its full length through the
             * faces it meets if the hinge's voxel is homogeneous and the
             * segment ends in its neighbourhood; otherwise, and in the EPID,
             * it stops at the face. */
            if (p->zone == Z_CT) through = leg_through(c, p->x, p->u, p->cell, s2, ecell);
            if (!through) { s2 = sb2; crossed = 1; }
        }
        for (int a = 0; a < 3; a++) p->x[a] += s2 * p->u[a];
        if (track) c->probe->path[c->probe->hidx] += s1 + s2;
        double dE = dEt * ((s1 + s2) / sE);
        double Tn = T - dE;
        /* a hard-event step that ran its full length ends at the tentative
         * event, which consumes the optical depth; otherwise spend the path */
        const int at_event = (lim == 1 && !crossed);
        if (at_event) p->tau = 0.0; else p->tau -= (s1 + s2) * Sh;
        o_part here = *p;
        here.cell[0] = hcell[0]; here.cell[1] = hcell[1]; here.cell[2] = hcell[2];
        if (Tn <= tstop) {
            /* the particle stops at its hinge point */
            probe_end(c, p, hinge);
            deposit(c, &here, hinge, hcell[0], dE + Tn);
            if (p->type == P_POSITRON) {
                p->x[0] = hinge[0]; p->x[1] = hinge[1]; p->x[2] = hinge[2];
                p->cell[0] = hcell[0]; p->cell[1] = hcell[1]; p->cell[2] = hcell[2];
                annihilate(c, p);
            }
            return;
        }
        if (through) {
            /* the step's energy split by path length over the voxels of the
             * second segment (the first segment and the second's first piece
             * lie in the hinge's voxel); each piece deposited at its midpoint,
             * the last in the voxel where the step ends */
            int segcell[O_MAXFACES + 1][3];
            double seglen[O_MAXFACES + 1];
            const int nseg = leg_walk(c, hinge, p->u, hcell, s2, segcell, seglen);
            for (int a = 0; a < 3; a++) segcell[nseg - 1][a] = ecell[a];
            double left = dE, at = 0.0;
            for (int k = 0; k < nseg; k++) {
                double e = (k + 1 < nseg) ? dE * ((k == 0 ? s1 + seglen[0] : seglen[k]) / (s1 + s2)) : left;
                double mp[3];
                for (int a = 0; a < 3; a++) mp[a] = hinge[a] + (at + 0.5 * seglen[k]) * p->u[a];
                o_part piece = *p;
                for (int a = 0; a < 3; a++) piece.cell[a] = segcell[k][a];
                deposit(c, &piece, k == 0 ? hinge : mp, piece.cell[0], e);
                left -= e;
                at += seglen[k];
            }
            for (int a = 0; a < 3; a++) p->cell[a] = ecell[a];
        } else {
            deposit(c, &here, hinge, hcell[0], dE);
        }
        p->E = Tn;
        if (crossed) {
            if (p->zone == Z_CT) {
                p->cell[ax2] += (p->u[ax2] > 0.0) ? 1 : -1;
                int n[3] = {P->nx, P->ny, P->nz};
                if (p->cell[ax2] < 0 || p->cell[ax2] >= n[ax2]) { transfer_to_epid(c, p); return; }
            } else {
                if (ax2 != 0) { escape(c, p, p->E + rest_extra(p)); return; }
                int nl = layer + (p->u[2] < 0.0 ? 1 : -1);
                if (nl < 0 || nl >= P->n_layers) { escape(c, p, p->E + rest_extra(p)); return; }
                p->cell[0] = nl;
            }
            continue;
        }
        if (at_event) {
            double Sn_m = rho * orc_sigma_moller(m, Tn, P->wcc);
            double Sn_b = rho * orc_sigma_brem(m, Tn, P->wcb);
            if (!(rng_u(&p->rng) * Sh < Sn_m + Sn_b)) continue;        /* delta event */
            const int is_moller = rng_u(&p->rng) * (Sn_m + Sn_b) < Sn_m;
            orc_probe* Q = c->probe;
            if (Q && p->prim && !Q->hard_done) {
                Q->hard_done = 1;
                if (Q->hard_T) Q->hard_T[Q->hidx] = Tn;
                if (Q->hard_type) Q->hard_type[Q->hidx] = is_moller ? 0 : 1;
            }
            if (is_moller) {
                c->cnt[C_MOLLER]++;
                double eps = sample_moller_eps(&p->rng, Tn, P->wcc);
                double phi = 2.0 * O_PI * rng_u(&p->rng);
                double W = eps * Tn, Tp = Tn - W;
                double cs = sqrt(W * (Tn + 2.0 * O_MC2) / (Tn * (W + 2.0 * O_MC2)));
                double cp = sqrt(Tp * (Tn + 2.0 * O_MC2) / (Tn * (Tp + 2.0 * O_MC2)));
                double us[3] = {p->u[0], p->u[1], p->u[2]};
                const double u0[3] = {p->u[0], p->u[1], p->u[2]};
                rotate(us, cs, phi);
                rotate(p->u, cp, phi + O_PI);
                if (Q) {
                    /* momentum balance of the free-electron collision */
                    double p0 = p_of_T(Tn), pw = p_of_T(W), pt = p_of_T(Tp), r2 = 0.0;
                    for (int a = 0; a < 3; a++) {
                        double d = p0 * u0[a] - pw * us[a] - pt * p->u[a];
                        r2 += d * d;
                    }
                    probe_max(fabs(u0[2]) > 0.99999 ? &Q->polar_dev : &Q->moller_dev, sqrt(r2) / p0);
                    probe_unit(c, us);
                    probe_unit(c, p->u);
                    Q->n_moller++;
                }
                emit_charged(c, p, P_ELECTRON, W, us, 0, layer);
                p->E = Tp;
            } else {
                c->cnt[C_BREM]++;
                double k = P->wcb * exp(rng_u(&p->rng) * log(Tn / P->wcb));
                o_part g;
                make_child(p, &g, P_PHOTON, 0);
                g.u[0] = p->u[0]; g.u[1] = p->u[1]; g.u[2] = p->u[2];
                g.E = k;
                if (Q) {
                    double r2 = 0.0;
                    for (int a = 0; a < 3; a++) r2 += (g.u[a] - p->u[a]) * (g.u[a] - p->u[a]);
                    probe_max(&Q->brem_dev, sqrt(r2));
                    if ((int64_t)Q->n_brem < Q->cap && Q->brem_x) Q->brem_x[Q->n_brem] = log(k / P->wcb) / log(Tn / P->wcb);
                    Q->n_brem++;
                }
                c->cnt[C_PHOTONS2]++;
                push(c, &g);
                p->E = Tn - k;
            }
            if (p->E <= tstop) {
                probe_end(c, p, p->x);
                deposit(c, p, p->x, layer, p->E);
                if (p->type == P_POSITRON) annihilate(c, p);
                return;
            }
        }
    }
    c->e_lost += p->E + rest_extra(p);
    c->cnt[C_LOST]++;
    if (c->probe && p->type == P_POSITRON) c->probe->n_pos_escape++;
}

/* ------------------------------------------------------------------------ */
/* Source (Sec. 2.1.1 with the jaw/MLC transport replaced by an ideal        */
/* aperture): rectangle chosen with weight MU_k x area, point uniform in it  */
/* at the isocentre plane, direction from the point source.                  */
/* ------------------------------------------------------------------------ */
/* Source rectangles at the isocentre plane: per segment and leaf pair (in
 * that order), within the jaws, the part of the pair left of the opening,
 * the opening, the part right of it (a closed pair is one part).  Openings
 * weigh MU x area; closed parts MU x T x area with T the leaf transmission
 * (absent when T = 0).  Returns whether any opening exists. */
static void add_rect(o_ctx* c, int* n, double* acc, double x0, double x1, double y0, double y1, double w,
                     int flag) {
    if (!(x1 > x0) || !(y1 > y0) || !(w > 0.0)) return;
    *acc += w * (x1 - x0) * (y1 - y0);
    c->rect[4 * *n] = x0; c->rect[4 * *n + 1] = x1; c->rect[4 * *n + 2] = y0; c->rect[4 * *n + 3] = y1;
    c->rflag[*n] = flag;
    c->cdf[*n] = *acc;
    (*n)++;
}

/* Half-width of the largest field at the isocentre plane (40 x 40 cm). */
#define O_FIELD_HALF 20.0

/* Effective opening [lo, hi] of pair j in segment k: the leaf tips moved
 * apart by half the leaf gap each, for a pair whose leaves are apart; a pair
 * whose tips meet or cross is closed (returns 0). */
static int pair_opening(const orc_problem* P, int k, int j, double* lo, double* hi) {
    const double* lf = P->leaves + 2 * ((size_t)k * P->n_pairs + j);
    if (!(lf[1] > lf[0])) return 0;
    *lo = lf[0] - 0.5 * P->leaf_gap;
    *hi = lf[1] + 0.5 * P->leaf_gap;
    return 1;
}

static int cmp_double(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Sorted distinct values of v[0..n) that lie strictly inside (lo, hi),
 * framed by lo and hi; returns the count. */
static int breakpoints(double lo, double hi, const double* v, int n, double* out) {
    int m = 0;
    out[m++] = lo;
    for (int i = 0; i < n; i++)
        if (v[i] > lo && v[i] < hi) out[m++] = v[i];
    out[m++] = hi;
    qsort(out + 1, (size_t)(m - 2), sizeof(double), cmp_double);
    int u = 1;
    for (int i = 1; i < m; i++)
        if (out[i] != out[u - 1]) out[u++] = out[i];
    return u;
}

/* Source of Sec. 2.1.1 with the collimators as fluence filters (the paper
 * transports the beam through jaws and MLC; no head model is available, so
 * this is the stated reading).  Per MU, the fluence at a point (X, Y) of the
 * isocentre plane inside the largest field and the MLC's extent is
 *   (leaf factor) x (jaw factor),
 * leaf factor = 1 inside the effective opening of the point's pair, else the
 * leaf transmission; within half the tongue-and-groove width of the boundary
 * between two pairs the opening is the intersection of both pairs' openings;
 * jaw factor = 1 inside the segment's jaws, else the jaw transmission.  Each
 * segment, pair, band of Y and interval of X on which both factors are
 * constant is one rectangle, weighted by MU x factors x area, in that order
 * (segments, pairs, increasing Y, increasing X). */
static int build_source(o_ctx* c) {
    const orc_problem* P = c->P;
    const double C = O_FIELD_HALF, w = P->tg_width;
    int nmax = 25 * P->n_seg * P->n_pairs;
    c->rect = (double*)malloc(sizeof(double) * 4 * (size_t)(nmax > 0 ? nmax : 1));
    c->rflag = (int*)malloc(sizeof(int) * (size_t)(nmax > 0 ? nmax : 1));
    c->cdf = (double*)malloc(sizeof(double) * (size_t)(nmax > 0 ? nmax : 1));
    /* collimator slabs (leaves and jaws as tungsten of the stated thickness):
     * every rectangle of the field weighs MU x area, and its flags say which
     * slabs its photons cross; without slabs the fluence factors apply */
    const int slab = P->leaf_thick > 0.0 || P->jaw_thick > 0.0;
    double acc = 0.0;
    int n = 0, open = 0;
    for (int k = 0; k < P->n_seg; k++) {
        const double* jw = P->jaws + 4 * k;
        const double mu = P->mu[k];
        if (!(mu > 0.0)) continue;
        const double jx0 = fmax(jw[0], -C), jx1 = fmin(jw[1], C);
        const double jy0 = fmax(jw[2], -C), jy1 = fmin(jw[3], C);
        for (int j = 0; j < P->n_pairs; j++) {
            const double e0 = P->pair_edges[j], e1 = P->pair_edges[j + 1];
            const double* lf = P->leaves + 2 * ((size_t)k * P->n_pairs + j);
            /* the physical aperture, for the field size of Eq. 1 */
            if (fmin(lf[1], jw[1]) > fmax(lf[0], jw[0]) && fmin(e1, jw[3]) > fmax(e0, jw[2])) open = 1;
            const double ya = fmax(e0, -C), yb = fmin(e1, C);
            if (!(yb > ya)) continue;
            double ycut[4] = {jy0, jy1, e0 + 0.5 * w, e1 - 0.5 * w}, yb_[6];
            const int ny = breakpoints(ya, yb, ycut, (w > 0.0) ? 4 : 2, yb_);
            for (int b = 0; b + 1 < ny; b++) {
                const double y0 = yb_[b], y1 = yb_[b + 1], ym = 0.5 * (y0 + y1);
                double lo = 0.0, hi = 0.0;
                int has = pair_opening(P, k, j, &lo, &hi);
                int nb = -1;                      /* the neighbour sharing a tongue-and-groove strip */
                if (w > 0.0 && j > 0 && ym < e0 + 0.5 * w) nb = j - 1;
                if (w > 0.0 && j + 1 < P->n_pairs && ym > e1 - 0.5 * w) nb = j + 1;
                if (has && nb >= 0) {
                    double lo2, hi2;
                    if (pair_opening(P, k, nb, &lo2, &hi2)) {
                        lo = fmax(lo, lo2);
                        hi = fmin(hi, hi2);
                        has = hi > lo;
                    } else {
                        has = 0;
                    }
                }
                const int in_jaw_y = ym >= jy0 && ym <= jy1;
                double xcut[4] = {jx0, jx1, lo, hi}, xb[6];
                const int nx = breakpoints(-C, C, xcut, has ? 4 : 2, xb);
                for (int a = 0; a + 1 < nx; a++) {
                    const double x0 = xb[a], x1 = xb[a + 1], xm = 0.5 * (x0 + x1);
                    const int in_leaf = has && xm >= lo && xm <= hi;
                    const int in_jaw = in_jaw_y && xm >= jx0 && xm <= jx1;
                    double leaf, jaw;
                    if (slab) {
                        leaf = (in_leaf || P->leaf_thick > 0.0) ? 1.0 : 0.0;
                        jaw = (in_jaw || P->jaw_thick > 0.0) ? 1.0 : 0.0;
                    } else {
                        leaf = in_leaf ? 1.0 : P->leaf_trans;
                        jaw = in_jaw ? 1.0 : P->jaw_trans;
                    }
                    add_rect(c, &n, &acc, x0, x1, y0, y1, mu * leaf * jaw,
                             slab ? ((in_leaf ? 0 : 1) | (in_jaw ? 0 : 2)) : 0);
                }
            }
        }
    }
    c->n_rect = n;
    if (!(acc > 0.0)) return 0;
    for (int i = 0; i < n; i++) c->cdf[i] /= acc;
    return open;
}

/* Draws of a primary: rectangle (1), X (1), Y (1), then the spectrum.
 * Returns the rectangle's slab flags. */
static int sample_source(const o_ctx* c, o_rng* r, double* X, double* Y, double* E) {
    const orc_problem* P = c->P;
    /* rectangle: first index whose cumulative weight exceeds the draw */
    double xi = rng_u(r);
    int lo = 0, hi = c->n_rect - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (xi < c->cdf[mid]) hi = mid; else lo = mid + 1;
    }
    const double* q = c->rect + 4 * lo;
    *X = q[0] + (q[1] - q[0]) * rng_u(r);
    *Y = q[2] + (q[3] - q[2]) * rng_u(r);
    *E = (P->mono_e > 0.0) ? P->mono_e : sample_spectrum(r, P->e_max, P->pcut);
    return c->rflag[lo];
}

/* Photon transport through a laterally infinite tungsten slab between the
 * beam-frame planes Z = zt (top) and Z = zb < zt: flights against mu_W(E),
 * Compton scattering (Klein-Nishina, the photon goes on), photoelectric
 * absorption and pair production absorbed in the collimator (their electrons
 * and annihilation photons do not leave the head; stated reading).  x (on or
 * above the top plane), u, E in the beam frame; returns 1 with the state at
 * the bottom plane if the photon leaves there, 0 if it is absorbed, falls
 * below the photon cutoff or leaves through the top. */
static int slab_transport(const orc_problem* P, o_rng* r, double x[3], double u[3], double* E, double zt, double zb,
                          int* collided) {
    for (int f = 0; f < P->max_steps; f++) {
        double mu[3];
        orc_mu_photon(O_MAT_W, *E, mu);
        const double tot = O_W_RHO * (mu[0] + mu[1] + mu[2]);
        rng_align(r);
        const double s = -log(rng_u(r)) / tot;
        double d = INFINITY;
        if (u[2] < 0.0) d = (zb - x[2]) / u[2];
        else if (u[2] > 0.0) d = (zt - x[2]) / u[2];
        if (!(s < d)) {
            if (!(u[2] < 0.0)) return 0;
            for (int a = 0; a < 3; a++) x[a] += d * u[a];
            x[2] = zb;
            return 1;
        }
        for (int a = 0; a < 3; a++) x[a] += s * u[a];
        const double xi = rng_u(r);
        if (!(xi * (mu[0] + mu[1] + mu[2]) < mu[0])) return 0;     /* photoelectric or pair */
        double eps, ct;
        sample_kn(r, *E, &eps, &ct);
        rotate(u, ct, 2.0 * O_PI * rng_u(r));
        *E *= eps;
        *collided = 1;
        if (*E < P->pcut) return 0;
    }
    return 0;
}

/* Phase space 2 of Sec. 2.1.1 with the collimators as tungsten slabs: photons
 * of the open-beam source (phase space 1) are drawn, with the history's own
 * stream, until one leaves the jaw and leaf slabs it crosses (a rectangle's
 * flags: bit 1 outside the jaws, bit 0 behind a closed leaf; jaws above the
 * MLC); that photon is the history.  Returns 1 with its beam-frame position
 * x (the source, or the bottom of the last slab crossed), direction u,
 * energy, the isocentre-plane point (X, Y) of its source ray, whether it
 * scattered in a slab and the number of source photons drawn; 0 if
 * O_PS1_CAP draws all ended in the collimators. */
#define O_PS1_CAP 100000
static int sample_ps2(const o_ctx* c, o_rng* r, double* X, double* Y, double* E, double x[3], double u[3],
                      int* collided, int* n_ps1) {
    const orc_problem* P = c->P;
    for (int k = 0; k < O_PS1_CAP; k++) {
        const int flag = sample_source(c, r, X, Y, E);
        *n_ps1 = k + 1;
        const double nb = sqrt(*X * *X + *Y * *Y + P->sad * P->sad);
        x[0] = 0.0; x[1] = 0.0; x[2] = P->sad;
        u[0] = *X / nb; u[1] = *Y / nb; u[2] = -P->sad / nb;
        *collided = 0;
        if (flag & 2) {
            const double zt = P->sad - O_JAW_TOP, t = (zt - x[2]) / u[2];
            for (int a = 0; a < 3; a++) x[a] += t * u[a];
            x[2] = zt;
            if (!slab_transport(P, r, x, u, E, zt, zt - P->jaw_thick, collided)) continue;
        }
        if (flag & 1) {
            const double zt = P->sad - O_MLC_TOP, t = (zt - x[2]) / u[2];
            for (int a = 0; a < 3; a++) x[a] += t * u[a];
            x[2] = zt;
            if (!slab_transport(P, r, x, u, E, zt, zt - P->leaf_thick, collided)) continue;
        }
        return 1;
    }
    return 0;
}

/* Transport every particle on the stack, and their descendants, to the end. */
static void drain(o_ctx* c) {
    while (c->sp > 0) {
        o_part q = c->stack[--c->sp];
        if (q.type == P_PHOTON) {
            if (q.zone == Z_CT) photon_ct(c, &q); else photon_epid(c, &q);
        } else {
            electron(c, &q);
        }
    }
}

static void run_history(o_ctx* c, uint64_t h, uint64_t seed) {
    c->hist = h;
    o_part p;
    memset(&p, 0, sizeof(p));
    p.type = P_PHOTON;
    p.rng.key[0] = (uint32_t)seed; p.rng.key[1] = (uint32_t)(seed >> 32);
    p.rng.ord = 0; p.rng.hlo = (uint32_t)h; p.rng.hhi = (uint32_t)(h >> 32);
    p.rng.d = 0; p.rng.cvalid = 0;
    double X, Y, sb[3], ub[3];
    int n_ps1;
    if (!sample_ps2(c, &p.rng, &X, &Y, &p.E, sb, ub, &p.collided, &n_ps1)) return;
    c->e_src += p.E;
    to_patient(c, sb, p.x);
    to_patient_dir(c, ub, p.u);
    enter_world(c, &p);
    drain(c);
}

/* ------------------------------------------------------------------------ */
/* Driver: threads own disjoint sub-tallies (b = h mod B), so the tally is    */
/* independent of the thread count.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    o_ctx local; uint64_t seed, h0, n; int tid, nthreads;
} o_job;

/* Macro-cells of M^3 voxels (the last ones along an axis may be partial);
 * each keeps the largest density of its non-bone and of its bone voxels, the
 * local Woodcock majorant. */
static void ctx_macro_grid(o_ctx* c, int M) {
    const orc_problem* P = c->P;
    const int n[3] = {P->nx, P->ny, P->nz};
    free(c->mg_low);
    free(c->mg_bone);
    c->mgM = M;
    for (int a = 0; a < 3; a++) c->mg[a] = (n[a] + M - 1) / M;
    size_t ncell = (size_t)c->mg[0] * c->mg[1] * c->mg[2];
    c->mg_low = (double*)calloc(ncell, sizeof(double));
    c->mg_bone = (double*)calloc(ncell, sizeof(double));
    for (int iz = 0; iz < P->nz; iz++)
        for (int iy = 0; iy < P->ny; iy++)
            for (int ix = 0; ix < P->nx; ix++) {
                double rho; int m;
                orc_hu_to_rho_mat(P->hu[((size_t)iz * P->ny + iy) * P->nx + ix], &rho, &m);
                size_t cc = ((size_t)(iz / M) * c->mg[1] + iy / M) * c->mg[0] + ix / M;
                double* tgt = (m == 3) ? &c->mg_bone[cc] : &c->mg_low[cc];
                if (rho > *tgt) *tgt = rho;
            }
}

/* A voxel is homogeneous when it lies at least O_HOM_R voxels inside the CT
 * and the (2 O_HOM_R + 1)^3 box around it holds one material with HU values
 * (clamped to [-1024, 3071]) spanning at most O_HOM_SPAN: an electron step's
 * second segment may then run into that box with the voxel's own stopping
 * power.  The box minimum and maximum are taken one axis at a time (the
 * extremes of a box are the extremes of its rows' extremes); materials rise
 * with HU, so one material means the material of the minimum equals that of
 * the maximum. */
static int clamp_hu(int h) { return h < -1024 ? -1024 : (h > 3071 ? 3071 : h); }
static void ctx_homogeneity(o_ctx* c) {
    const orc_problem* P = c->P;
    const int n[3] = {P->nx, P->ny, P->nz};
    const size_t nv = (size_t)n[0] * n[1] * n[2];
    const size_t st[3] = {1, (size_t)n[0], (size_t)n[0] * n[1]};
    int* lo = (int*)malloc(sizeof(int) * nv);
    int* hi = (int*)malloc(sizeof(int) * nv);
    int* lo2 = (int*)malloc(sizeof(int) * nv);
    int* hi2 = (int*)malloc(sizeof(int) * nv);
    for (size_t v = 0; v < nv; v++) lo[v] = hi[v] = clamp_hu(P->hu[v]);
    for (int a = 0; a < 3; a++) {
        for (int iz = 0; iz < n[2]; iz++)
            for (int iy = 0; iy < n[1]; iy++)
                for (int ix = 0; ix < n[0]; ix++) {
                    const int idx[3] = {ix, iy, iz};
                    const size_t v = ((size_t)iz * n[1] + iy) * n[0] + ix;
                    int mn = lo[v], mx = hi[v];
                    for (int d = -O_HOM_R; d <= O_HOM_R; d++) {
                        const int k = idx[a] + d;
                        if (k < 0 || k >= n[a]) continue;
                        const size_t w = v + (ptrdiff_t)d * (ptrdiff_t)st[a];
                        if (lo[w] < mn) mn = lo[w];
                        if (hi[w] > mx) mx = hi[w];
                    }
                    lo2[v] = mn; hi2[v] = mx;
                }
        int* t;
        t = lo; lo = lo2; lo2 = t;
        t = hi; hi = hi2; hi2 = t;
    }
    c->hom = (unsigned char*)calloc(nv, 1);
    for (int iz = O_HOM_R; iz + O_HOM_R < n[2]; iz++)
        for (int iy = O_HOM_R; iy + O_HOM_R < n[1]; iy++)
            for (int ix = O_HOM_R; ix + O_HOM_R < n[0]; ix++) {
                const size_t v = ((size_t)iz * n[1] + iy) * n[0] + ix;
                double r; int m_lo, m_hi;
                orc_hu_to_rho_mat(lo[v], &r, &m_lo);
                orc_hu_to_rho_mat(hi[v], &r, &m_hi);
                c->hom[v] = (unsigned char)(m_lo == m_hi && hi[v] - lo[v] <= O_HOM_SPAN);
            }
    free(lo); free(hi); free(lo2); free(hi2);
}

static void ctx_geometry(o_ctx* c, const orc_problem* P) {
    memset(c, 0, sizeof(*c));
    c->P = P;
    double g = P->gantry_deg * O_PI / 180.0;
    c->ex[0] = cos(g); c->ex[1] = sin(g); c->ex[2] = 0.0;
    c->ey[0] = 0.0; c->ey[1] = 0.0; c->ey[2] = 1.0;
    c->ez[0] = sin(g); c->ez[1] = -cos(g); c->ez[2] = 0.0;
    double zs = P->sad - P->sid;
    double z = zs + 0.5 * P->layer_thick[P->sens_layer];
    for (int l = P->sens_layer - 1; l >= 0; l--) z += P->layer_thick[l];
    c->zplane[0] = z;
    for (int l = 0; l < P->n_layers; l++) c->zplane[l + 1] = c->zplane[l] - P->layer_thick[l];
    c->half_w[0] = 0.5 * P->npx * P->pitch;
    c->half_w[1] = 0.5 * P->npy * P->pitch;
    size_t nv = (size_t)P->nx * P->ny * P->nz;
    for (size_t i = 0; i < nv; i++) {
        double rho; int m;
        orc_hu_to_rho_mat(P->hu[i], &rho, &m);
        c->mat_present[m] = 1;
        if (rho > c->rho_max[m]) c->rho_max[m] = rho;
    }
    /* macro-cells of M^3 voxels, M the smallest power of two >= 4 whose
     * cells are at least 6 cm along every axis and number at most 4096 (any
     * majorant that bounds mu along the ray gives the same real collisions;
     * the size only trades virtual collisions against cell steps) */
    int n[3] = {P->nx, P->ny, P->nz};
    double vmin = fmin(P->vox[0], fmin(P->vox[1], P->vox[2]));
    int M = 4;
    for (;;) {
        long cells = 1;
        for (int a = 0; a < 3; a++) cells *= (n[a] + M - 1) / M;
        /* (a cell as large as the whole CT also ends the search) */
        if (cells <= 4096 && (M * vmin >= 6.0 || (M >= n[0] && M >= n[1] && M >= n[2]))) break;
        M *= 2;
    }
    ctx_macro_grid(c, M);
}

static void ctx_free(o_ctx* c) {
    free(c->mg_low);
    free(c->mg_bone);
    free(c->hom);
    c->mg_low = c->mg_bone = NULL;
    c->hom = NULL;
}

static void* worker(void* arg) {
    o_job* J = (o_job*)arg;
    o_ctx* c = &J->local;
    uint64_t B = (uint64_t)c->P->n_batches;
    for (uint64_t i = 0; i < J->n; i++) {
        uint64_t h = J->h0 + i;
        if ((int)((h % B) % (uint64_t)J->nthreads) != J->tid) continue;
        run_history(c, h, J->seed);
    }
    return NULL;
}

int orc_run(const orc_problem* P, uint64_t seed, uint64_t hist_begin, uint64_t n_hist, int n_threads,
            orc_result* R) {
    if (!P || !R || !R->tally || P->n_layers < 1 || P->n_layers > O_MAXL || P->n_batches < 1) return 1;
    o_ctx base;
    ctx_geometry(&base, P);
    ctx_homogeneity(&base);
    if (!build_source(&base)) { free(base.rect); free(base.rflag); free(base.cdf); ctx_free(&base); return 2; }
    if (n_threads < 1) n_threads = 1;
    if (n_threads > P->n_batches) n_threads = P->n_batches;
    o_job* jobs = (o_job*)calloc((size_t)n_threads, sizeof(o_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    const size_t nvox = (size_t)P->nx * P->ny * P->nz;
    for (int t = 0; t < n_threads; t++) {
        jobs[t].local = base;
        jobs[t].local.tally = R->tally;
        jobs[t].local.vox = R->vox ? (double*)calloc(nvox, sizeof(double)) : NULL;
        jobs[t].local.stack = NULL; jobs[t].local.sp = 0; jobs[t].local.cap = 0;
        jobs[t].seed = seed; jobs[t].h0 = hist_begin; jobs[t].n = n_hist;
        jobs[t].tid = t; jobs[t].nthreads = n_threads;
    }
    for (int t = 1; t < n_threads; t++) pthread_create(&th[t], NULL, worker, &jobs[t]);
    worker(&jobs[0]);
    for (int t = 1; t < n_threads; t++) pthread_join(th[t], NULL);
    for (int t = 0; t < n_threads; t++) {
        o_ctx* l = &jobs[t].local;
        R->e_src += l->e_src; R->e_ct += l->e_ct; R->e_esc += l->e_esc; R->e_lost += l->e_lost;
        for (int k = 0; k < O_MAXL; k++) R->e_epid[k] += l->e_epid[k];
        for (int k = 0; k < C_NCOUNT; k++) R->counters[k] += l->cnt[k];
        if (l->vox) {
            for (size_t v = 0; v < nvox; v++) R->vox[v] += l->vox[v];
            free(l->vox);
        }
        free(l->stack);
    }
    free(jobs); free(th); free(base.rect); free(base.rflag); free(base.cdf);
    ctx_free(&base);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Test hooks: single samplers exposed for the CPU pins.                     */
/* ------------------------------------------------------------------------ */
static void hook_rng(o_rng* r, uint64_t seed, uint64_t h) {
    memset(r, 0, sizeof(*r));
    r->key[0] = (uint32_t)seed; r->key[1] = (uint32_t)(seed >> 32);
    r->hlo = (uint32_t)h; r->hhi = (uint32_t)(h >> 32);
}

void orc_uniforms(uint64_t seed, uint64_t h, uint32_t ord, uint32_t n, double* out) {
    o_rng r; hook_rng(&r, seed, h); r.ord = ord;
    for (uint32_t i = 0; i < n; i++) out[i] = rng_u(&r);
}

void orc_sample_kn_many(double E, uint64_t seed, uint64_t n, double* eps, double* cost) {
    for (uint64_t i = 0; i < n; i++) {
        o_rng r; hook_rng(&r, seed, i);
        sample_kn(&r, E, &eps[i], &cost[i]);
    }
}

void orc_sample_spectrum_many(double emax, double ecut, uint64_t seed, uint64_t n, double* out) {
    for (uint64_t i = 0; i < n; i++) {
        o_rng r; hook_rng(&r, seed, i);
        out[i] = sample_spectrum(&r, emax, ecut);
    }
}

void orc_sample_moller_many(double T, double wcc, uint64_t seed, uint64_t n, double* eps) {
    for (uint64_t i = 0; i < n; i++) {
        o_rng r; hook_rng(&r, seed, i);
        eps[i] = sample_moller_eps(&r, T, wcc);
    }
}

void orc_sample_ms_many(double G, uint64_t seed, uint64_t n, double* cost) {
    double A = orc_wentzel_A(G);
    for (uint64_t i = 0; i < n; i++) {
        o_rng r; hook_rng(&r, seed, i);
        double mu = (G > 0.0) ? sample_ms_mu(A, rng_u(&r)) : 0.0;
        cost[i] = 1.0 - 2.0 * mu;
    }
}

/* CSDA path length of an electron in an unbounded medium of material m with
 * hard events and deflections switched off: the step rule alone. */
double orc_csda_path(int m, double rho, double T0, double ecut, double wcc, double wcb, double step_frac) {
    double T = T0, path = 0.0;
    const double tstop = ecut + O_TSTOP;
    for (int i = 0; i < 1000000 && T > tstop; i++) {
        double dEt = step_frac * T;
        if (T - dEt < tstop) dEt = T - ecut;
        double Tm = T - 0.5 * dEt;
        double L = rho * (orc_lcol(m, Tm, wcc) + orc_lrad_soft(m, Tm, wcb));
        path += dEt / L;
        T -= dEt;
    }
    return path;
}

/* First real photon interaction along one fixed ray through the CT of P:
 * for n photons of energy E starting at `start` (patient frame) along `dir`,
 * record the flat voxel index (-1 if none before leaving the box) and the
 * interaction type (0 Compton, 1 photoelectric, 2 pair).  macro_M > 0 sets
 * the macro-cell size of the majorant grid (0: the default rule). */
void orc_first_interaction(const orc_problem* P, double E, const double start[3], const double dir[3],
                           uint64_t seed, uint64_t n, int macro_M, int64_t* vox, int32_t* type) {
    o_ctx c;
    ctx_geometry(&c, P);
    if (macro_M > 0) ctx_macro_grid(&c, macro_M);
    for (uint64_t i = 0; i < n; i++) {
        o_rng r; hook_rng(&r, seed, i);
        double x[3] = {start[0], start[1], start[2]};
        vox[i] = -1; type[i] = -1;
        for (int f = 0; f < 100000; f++) {
            int idx[3];
            double Sc;
            if (!ct_flight(&c, x, dir, E, &r, idx, &Sc)) break;
            double rho; int m;
            ct_props(&c, idx, &rho, &m);
            double mu[3];
            orc_mu_photon(m, E, mu);
            double tot = mu[0] + mu[1] + mu[2];
            if (!(rng_u(&r) * Sc < rho * tot)) continue;
            double xi = rng_u(&r);
            vox[i] = ((int64_t)idx[2] * P->ny + idx[1]) * P->nx + idx[0];
            type[i] = (xi * tot < mu[0]) ? 0 : (xi * tot < mu[0] + mu[1]) ? 1 : 2;
            break;
        }
    }
    ctx_free(&c);
}

/* Histories h0 .. h0+n-1 whose primary is the probe's particle (instead of a
 * source sample), transported by the same code as orc_run with the probe
 * recording.  A photon primary enters the world along its line (CT box entry,
 * or straight to the EPID when the line misses the CT); a charged primary must
 * start inside the CT.  One thread; R accumulates as in orc_run (a positron
 * primary's source energy includes its rest energy 2 mc^2). */
int orc_pencil(const orc_problem* P, orc_probe* Q, uint64_t seed, uint64_t h0, uint64_t n, orc_result* R) {
    if (!P || !Q || !R || !R->tally || P->n_layers < 1 || P->n_layers > O_MAXL || P->n_batches < 1) return 1;
    if (Q->type < P_PHOTON || Q->type > P_POSITRON || !(Q->E > 0.0)) return 1;
    o_ctx c;
    ctx_geometry(&c, P);
    ctx_homogeneity(&c);
    if (Q->macro_M > 0) ctx_macro_grid(&c, Q->macro_M);
    c.tally = R->tally;
    c.vox = R->vox;
    c.probe = Q;
    const int nn[3] = {P->nx, P->ny, P->nz};
    int cell[3];
    for (int a = 0; a < 3; a++) {
        cell[a] = (int)floor((Q->x[a] - P->origin[a]) / P->vox[a]);
        if (Q->type != P_PHOTON && (cell[a] < 0 || cell[a] >= nn[a])) { ctx_free(&c); return 3; }
    }
    for (uint64_t i = 0; i < n; i++) {
        const uint64_t h = h0 + i;
        c.hist = h;
        Q->hidx = (int64_t)i;
        Q->first_done = Q->pix_done = Q->hard_done = 0;
        if (Q->path) Q->path[i] = 0.0;
        if (Q->hard_T) Q->hard_T[i] = -1.0;
        if (Q->hard_type) Q->hard_type[i] = -1;
        if (Q->first_layer) Q->first_layer[i] = -2;
        if (Q->first_pixel) Q->first_pixel[i] = -1;
        if (Q->first_pos) Q->first_pos[3 * i] = Q->first_pos[3 * i + 1] = Q->first_pos[3 * i + 2] = NAN;
        if (Q->end_pos) Q->end_pos[3 * i] = Q->end_pos[3 * i + 1] = Q->end_pos[3 * i + 2] = NAN;
        o_part p;
        memset(&p, 0, sizeof(p));
        p.type = Q->type;
        p.prim = 1;
        p.rng.key[0] = (uint32_t)seed; p.rng.key[1] = (uint32_t)(seed >> 32);
        p.rng.hlo = (uint32_t)h; p.rng.hhi = (uint32_t)(h >> 32);
        p.E = Q->E;
        c.e_src += Q->E + rest_extra(&p);
        for (int a = 0; a < 3; a++) { p.x[a] = Q->x[a]; p.u[a] = Q->u[a]; }
        if (Q->type == P_PHOTON) {
            enter_world(&c, &p);
        } else {
            p.zone = Z_CT;
            for (int a = 0; a < 3; a++) p.cell[a] = cell[a];
            if (Q->type == P_POSITRON) Q->n_pos_born++;
            push(&c, &p);
        }
        drain(&c);
    }
    R->e_src += c.e_src; R->e_ct += c.e_ct; R->e_esc += c.e_esc; R->e_lost += c.e_lost;
    for (int k = 0; k < O_MAXL; k++) R->e_epid[k] += c.e_epid[k];
    for (int k = 0; k < C_NCOUNT; k++) R->counters[k] += c.cnt[k];
    free(c.stack);
    ctx_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Radiological thickness (Sec. 2.2, step 1): exact Siddon (1985) ray sum     */
/* t = sum_v rho_v l_v from the source to each requested pixel centre.        */
/* ------------------------------------------------------------------------ */
static int cmp_d(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

double orc_siddon_ray(const orc_problem* P, const double p1[3], const double p2[3]) {
    int n[3] = {P->nx, P->ny, P->nz};
    double d[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double amin = 0.0, amax = 1.0;
    for (int a = 0; a < 3; a++) {
        double lo = P->origin[a], hi = P->origin[a] + n[a] * P->vox[a];
        if (d[a] != 0.0) {
            double a0 = (lo - p1[a]) / d[a], a1 = (hi - p1[a]) / d[a];
            amin = fmax(amin, fmin(a0, a1));
            amax = fmin(amax, fmax(a0, a1));
        } else if (p1[a] <= lo || p1[a] >= hi) {
            return 0.0;
        }
    }
    if (amin >= amax) return 0.0;
    size_t cap = (size_t)(n[0] + n[1] + n[2] + 8);
    double* al = (double*)malloc(sizeof(double) * cap);
    size_t k = 0;
    al[k++] = amin; al[k++] = amax;
    for (int a = 0; a < 3; a++) {
        if (d[a] == 0.0) continue;
        for (int i = 0; i <= n[a]; i++) {
            double av = (P->origin[a] + i * P->vox[a] - p1[a]) / d[a];
            if (av > amin && av < amax) al[k++] = av;
        }
    }
    qsort(al, k, sizeof(double), cmp_d);
    double t = 0.0;
    for (size_t i = 0; i + 1 < k; i++) {
        double am = 0.5 * (al[i] + al[i + 1]);
        int idx[3], ok = 1;
        for (int a = 0; a < 3; a++) {
            idx[a] = (int)floor((p1[a] + am * d[a] - P->origin[a]) / P->vox[a]);
            if (idx[a] < 0 || idx[a] >= n[a]) ok = 0;
        }
        if (!ok) continue;
        double rho; int m;
        int hu = P->hu[((size_t)idx[2] * P->ny + idx[1]) * P->nx + idx[0]];
        orc_hu_to_rho_mat(hu, &rho, &m);
        t += rho * (al[i + 1] - al[i]) * len;
    }
    free(al);
    return t;
}

/* t for pixels (ix[i], iy[i]) of the EPID grid, rays from the source to the
 * pixel centres on the sensitive layer's mid-plane (SID from the source). */
void orc_tmap(const orc_problem* P, const int32_t* ix, const int32_t* iy, int64_t n, double* t) {
    o_ctx c;
    ctx_geometry(&c, P);
    double sb[3] = {0.0, 0.0, P->sad}, src[3];
    to_patient(&c, sb, src);
    for (int64_t i = 0; i < n; i++) {
        double pb[3] = {-c.half_w[0] + (ix[i] + 0.5) * P->pitch, -c.half_w[1] + (iy[i] + 0.5) * P->pitch,
                        P->sad - P->sid};
        double pp[3];
        to_patient(&c, pb, pp);
        t[i] = orc_siddon_ray(P, src, pp);
    }
    ctx_free(&c);
}

/* ------------------------------------------------------------------------ */
/* Global gamma index (Low et al. 1998) with a low-dose threshold, the form  */
/* of the paper's image comparisons (Sec. 2.3.3).  ref is the reference      */
/* image; ev is bilinearly interpolated on a sub-grid of step h (mm) over a  */
/* search radius rad (mm).  Returns the pass rate; gamma values go to gam    */
/* (NaN for pixels below the threshold).                                     */
/* ------------------------------------------------------------------------ */
static double bilin(const double* img, int nx, int ny, double fx, double fy) {
    if (fx < 0) fx = 0;
    if (fy < 0) fy = 0;
    if (fx > nx - 1) fx = nx - 1;
    if (fy > ny - 1) fy = ny - 1;
    int x0 = (int)floor(fx), y0 = (int)floor(fy);
    int x1 = x0 + 1 < nx ? x0 + 1 : x0, y1 = y0 + 1 < ny ? y0 + 1 : y0;
    double ax = fx - x0, ay = fy - y0;
    return (1 - ay) * ((1 - ax) * img[(size_t)y0 * nx + x0] + ax * img[(size_t)y0 * nx + x1]) +
           ay * ((1 - ax) * img[(size_t)y1 * nx + x0] + ax * img[(size_t)y1 * nx + x1]);
}

double orc_gamma(const double* ref, const double* ev, int nx, int ny, double pix_mm, double dd_frac,
                 double dta_mm, double thr_frac, double h_mm, double rad_mm, double* gam) {
    double rmax = 0.0;
    for (size_t i = 0; i < (size_t)nx * ny; i++) rmax = fmax(rmax, ref[i]);
    double ddabs = dd_frac * rmax;
    long npass = 0, neval = 0;
    int nsub = (int)ceil(rad_mm / h_mm);
    for (int y = 0; y < ny; y++) {
        for (int x = 0; x < nx; x++) {
            size_t i = (size_t)y * nx + x;
            if (ref[i] < thr_frac * rmax) { if (gam) gam[i] = NAN; continue; }
            neval++;
            double best = INFINITY;
            for (int sy = -nsub; sy <= nsub && best > 0.0; sy++) {
                for (int sx = -nsub; sx <= nsub; sx++) {
                    double dx = sx * h_mm, dy = sy * h_mm;
                    double r2 = dx * dx + dy * dy;
                    if (r2 > rad_mm * rad_mm) continue;
                    double dist2 = r2 / (dta_mm * dta_mm);
                    if (dist2 >= best) continue;
                    double v = bilin(ev, nx, ny, x + dx / pix_mm, y + dy / pix_mm);
                    double dv = (v - ref[i]) / ddabs;
                    double g2 = dist2 + dv * dv;
                    if (g2 < best) best = g2;
                }
            }
            double gv = sqrt(best);
            if (gam) gam[i] = gv;
            if (gv <= 1.0) npass++;
        }
    }
    return neval ? (double)npass / neval : 1.0;
}

/* Phase-space-2 samples of histories h0..h0+n-1 (sample_ps2): the final
 * source ray's isocentre-plane point (X, Y), the energy (NaN if none left
 * the collimators), whether it scattered in a slab and the source photons
 * drawn. */
int orc_sample_ps2_many(const orc_problem* P, uint64_t seed, uint64_t h0, uint64_t n, double* X, double* Y,
                        double* E, int32_t* collided, int32_t* n_ps1) {
    o_ctx c;
    ctx_geometry(&c, P);
    build_source(&c);
    if (c.n_rect == 0) { free(c.rect); free(c.rflag); free(c.cdf); ctx_free(&c); return 2; }
    for (uint64_t i = 0; i < n; i++) {
        o_rng r; hook_rng(&r, seed, h0 + i);
        double x[3], u[3];
        int coll = 0, k = 0;
        if (!sample_ps2(&c, &r, &X[i], &Y[i], &E[i], x, u, &coll, &k)) E[i] = NAN;
        collided[i] = coll;
        n_ps1[i] = k;
    }
    free(c.rect); free(c.rflag); free(c.cdf);
    ctx_free(&c);
    return 0;
}

/* Source samples (isocentre-plane X, Y and energy) of histories h0..h0+n-1. */
int orc_sample_source_many(const orc_problem* P, uint64_t seed, uint64_t h0, uint64_t n, double* X, double* Y,
                           double* E) {
    o_ctx c;
    ctx_geometry(&c, P);
    if (!build_source(&c)) { free(c.rect); free(c.rflag); free(c.cdf); ctx_free(&c); return 2; }
    for (uint64_t i = 0; i < n; i++) {
        o_rng r; hook_rng(&r, seed, h0 + i);
        sample_source(&c, &r, &X[i], &Y[i], &E[i]);
    }
    free(c.rect); free(c.rflag); free(c.cdf);
    ctx_free(&c);
    return 0;
}
