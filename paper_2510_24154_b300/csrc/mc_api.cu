// C ABI of the EPID transit Monte Carlo library (declared in archer_epid.h):
// context lifecycle, geometry and field set-up, the transport wave loop
// (driven from the host, or one CUDA graph whose waves loop on the device),
// statistics, the dose-to-signal correction and checkpointing.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <utility>
#include <vector>

#include "archer_epid.h"
#include "mc_aux.h"
#include "mc_device.cuh"
#include "physics_tables.h"

using mc::BankPtr;
using mc::Ctl;
using mc::FieldDev;
using mc::Params;

namespace {

// Host copy of one field: beam frame, source rectangles, Eq. 1 and how many
// of its histories have run (the next history index of its stream).
struct FieldHost {
    double ex[3], ey[3], ez[3], iso[3];
    double sad, sid, zface;
    int rect_off, n_rect;
    double s_eq, bbox_a, bbox_b;
    double leaf_t, jaw_t;     // collimator slab thicknesses, cm (0: ideal)
    uint64_t stream_base;     // random-stream id of the field's history 0 (f * 2^40)
    uint64_t hist_done;
};

// CTAs of 256 threads per SM each transport kernel is built for, measured
// best on the thorax workload: 4 (64 registers) for every kernel.
constexpr int kDefaultRegsVariant[4] = {4, 4, 4, 4};
constexpr size_t kHeadsBytes = sizeof(uint32_t) * mc::kNumBanks * mc::kHeadShards * mc::kHeadStride;
constexpr double kQuantaPerMeV = 2.56e8;
constexpr double kJoulePerMeV = 1.602176634e-13;
constexpr uint64_t kFieldStride = 1ull << 40;
constexpr unsigned int kMaxWaves = 1000000u;

}  // namespace

struct mc_ctx {
    int device = 0;
    int sm_count = 0;
    mc_config cfg{};
    std::string err;
    std::atomic<int> cancel{0};
    // physics tables
    mcphys::Tables tabs;
    float2* d_ptab = nullptr;
    float2* d_etab = nullptr;
    // transport launch shape per bank type
    int block = 256;
    int grid[mc::kNumBanks] = {0, 0, 0, 0};
    int minb[mc::kNumBanks] = {4, 4, 4, 4};
    int src_grid = 0;            // source kernel: 8 CTAs of 256 per SM, grid-stride
    // banks
    void* bank_mem = nullptr;
    BankPtr bank[mc::kNumBanks][2];
    uint32_t cap = 0;
    Ctl* d_ctl = nullptr;
    uint32_t* d_heads = nullptr;  // segment read counters of the input banks
    Ctl* h_ctl = nullptr;        // pinned
    // geometry
    bool has_geom = false;
    int nx = 0, ny = 0, nz = 0;
    double vox[3] = {0, 0, 0}, origin[3] = {0, 0, 0};
    int16_t* d_hu = nullptr;
    float* d_rho = nullptr;
    float* d_rho_hom = nullptr;       // CT densities, sign bit set on homogeneous voxels
    int* d_hom_tmp = nullptr;         // two int32 per voxel: scratch of the flag passes
    size_t nvox_alloc = 0;
    unsigned int* d_rho_max = nullptr;
    float* d_thr = nullptr;
    float rho_max[4] = {0, 0, 0, 0};
    float thr[3] = {0, 0, 0};
    int mgM = 4, mg[3] = {1, 1, 1};
    float2* d_mgrid = nullptr;
    mc_epid_desc epid{};
    double zp[MC_MAX_LAYERS + 1] = {};   // layer planes, beam frame, sensitive-layer centre at 0
    // fields
    std::vector<FieldHost> fields;
    bool has_field = false;
    FieldDev* d_fields = nullptr;
    unsigned long long* d_first = nullptr;
    float4* d_rect = nullptr;
    uint32_t* d_guide = nullptr;             // cut-point tables of the source CDFs
    double* d_cdf = nullptr;
    unsigned char* d_rflag = nullptr;   // per rectangle: collimator slabs its photons cross
    double* d_tmap = nullptr;    // [F][npix]
    bool has_lut = false;
    int lut_nt = 0;
    double* d_lut_t = nullptr;
    double* d_lut_ks = nullptr;  // [F][nt]: the k-table column at each field's s
    double k_scale = 1.0, t_offset = 0.0;
    // tallies
    unsigned long long* d_tally = nullptr;   // [F][B][npix]
    size_t tally_n = 0;
    unsigned long long* d_energy = nullptr;
    unsigned long long* d_events = nullptr;
    unsigned long long* d_vox = nullptr;     // patient dose: [nz][ny][nx], 2^-8 eV
    size_t vox_n = 0;
    // statistics scratch
    double* d_dose = nullptr;
    double* d_flu = nullptr;                 // source fluence on the EPID grid (mc_get_field_fluence)
    double* d_sigma = nullptr;
    double* d_nb = nullptr;
    unsigned long long* d_rsum = nullptr;    // region statistics: per-batch sums, then mean and error
    double* d_rstat = nullptr;
    double* d_u = nullptr;
    unsigned long long* d_maxbits = nullptr;
    double* d_part = nullptr;
    unsigned int* d_partc = nullptr;
    float* d_signal = nullptr;
    int last_waves = 0;
    uint32_t last_error = 0;
    double last_ms = 0;
    double last_kernel_ms[4] = {0, 0, 0, 0};
    uint32_t last_kernel_launches[4] = {0, 0, 0, 0};
    uint32_t last_launches = 0;
    std::vector<cudaEvent_t> ev_pool;
    cudaStream_t capture_stream = nullptr;
    // asynchronous (graph-driven) runs: the last run's start and end events,
    // whether its control block (waves, error bits) and time are still to be
    // read, and its launches per wave
    cudaEvent_t ev_run0 = nullptr, ev_run1 = nullptr;
    cudaGraph_t run_graph = nullptr;          // kept until the run is finalized: destroying an
    cudaGraphExec_t run_exec = nullptr;       // executable graph waits for it
    bool run_pending = false;
    uint32_t run_per_wave = 0;
    // pinned staging of the host data that calls copy without waiting
    FieldDev* h_fields = nullptr;              // [kMaxFields]
    unsigned long long* h_first = nullptr;     // [kMaxFields + 1]
    char* h_stage = nullptr;                   // source rectangles, CDF, k-table columns
    size_t h_stage_cap = 0;
    cudaEvent_t ev_stage = nullptr;            // recorded after the last copies out of h_stage
    // field buffers are kept while large enough: their capacities in elements
    size_t cap_guide = 0;
    size_t cap_tally = 0, cap_pix = 0, cap_parts = 0, cap_rect = 0, cap_cdf = 0, cap_tmap = 0, cap_lut_t = 0,
           cap_ks = 0, cap_rflag = 0;
};

namespace {

mc_status fail(mc_ctx* c, mc_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

#define CUDA_TRY(ctx, call)                                                                         \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

int npix(const mc_ctx* c) { return c->epid.npx * c->epid.npy; }
int nfields(const mc_ctx* c) { return static_cast<int>(c->fields.size()); }

bool is_electron(int t) { return t == mc::kElectronCT || t == mc::kElectronEPID; }

// Forgets the fields (the device buffers stay for reuse).
void clear_fields(mc_ctx* c) {
    c->tally_n = 0;
    c->fields.clear();
    c->has_field = false;
    c->has_lut = false;
}

void free_field_buffers(mc_ctx* c) {
    dfree(c->d_rect);
    dfree(c->d_guide);
    dfree(c->d_cdf);
    dfree(c->d_rflag);
    dfree(c->d_tmap);
    dfree(c->d_lut_t);
    dfree(c->d_lut_ks);
    dfree(c->d_dose);
    dfree(c->d_flu);
    dfree(c->d_sigma);
    dfree(c->d_part);
    dfree(c->d_partc);
    dfree(c->d_signal);
    dfree(c->d_tally);
    c->cap_tally = c->cap_pix = c->cap_parts = c->cap_rect = c->cap_cdf = c->cap_tmap = c->cap_lut_t = c->cap_ks = 0;
    c->cap_rflag = 0;
    c->cap_guide = 0;
    clear_fields(c);
}

// Device buffer p holds at least n elements (kept if it already does;
// otherwise replaced, contents lost).
template <typename T>
cudaError_t ensure(T*& p, size_t& cap, size_t n) {
    if (n <= cap && p) return cudaSuccess;
    dfree(p);
    cap = 0;
    const cudaError_t e = cudaMalloc(&p, sizeof(T) * (n > 0 ? n : 1));
    if (e == cudaSuccess) cap = n;
    return e;
}

// The bookkeeping of a pending graph-driven run: waits for its end, reads
// its control block and time.  Returns the run's device-side outcome
// (bank overflow, wave limit) once; the error bits stay in the stats.
void release_run_graph(mc_ctx* c) {
    if (c->run_exec) cudaGraphExecDestroy(c->run_exec);
    if (c->run_graph) cudaGraphDestroy(c->run_graph);
    c->run_exec = nullptr;
    c->run_graph = nullptr;
}

mc_status finalize_run(mc_ctx* c) {
    if (!c->run_pending) return MC_OK;
    c->run_pending = false;
    const cudaError_t e = cudaEventSynchronize(c->ev_run1);
    release_run_graph(c);
    CUDA_TRY(c, e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev_run0, c->ev_run1);
    const Ctl& h = *c->h_ctl;
    c->last_waves = static_cast<int>(h.waves);
    c->last_error = h.error;
    c->last_ms = ms;
    c->last_launches = c->run_per_wave * h.waves;
    for (int t = 0; t < 4; ++t) {
        c->last_kernel_ms[t] = 0.0;
        c->last_kernel_launches[t] = (is_electron(t) && !c->cfg.coupled) ? 0u : h.waves;
    }
    if (h.error) return fail(c, MC_ERR_OVERFLOW, "particle bank overflow");
    if (h.waves >= kMaxWaves) return fail(c, MC_ERR_TIMEOUT, "wave limit reached");
    return MC_OK;
}

// Work queued on stream s after this call runs after the pending run.
mc_status order_after_run(mc_ctx* c, cudaStream_t s) {
    if (c->run_pending) CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_run1, 0));
    return MC_OK;
}

mc_status clear_tally(mc_ctx* c, cudaStream_t s) {
    if (c->d_tally) CUDA_TRY(c, cudaMemsetAsync(c->d_tally, 0, c->tally_n * sizeof(unsigned long long), s));
    CUDA_TRY(c, cudaMemsetAsync(c->d_energy, 0, sizeof(unsigned long long) * mc::kNumEnergy, s));
    CUDA_TRY(c, cudaMemsetAsync(c->d_events, 0, sizeof(unsigned long long) * mc::kNumEvents, s));
    if (c->d_vox) CUDA_TRY(c, cudaMemsetAsync(c->d_vox, 0, c->vox_n * sizeof(unsigned long long), s));
    for (FieldHost& f : c->fields) f.hist_done = 0;
    return MC_OK;
}

void make_params(const mc_ctx* c, Params& P, uint64_t seed) {
    std::memset(&P, 0, sizeof(P));
    P.nx = c->nx; P.ny = c->ny; P.nz = c->nz;
    P.ox = static_cast<float>(c->origin[0]); P.oy = static_cast<float>(c->origin[1]);
    P.oz = static_cast<float>(c->origin[2]);
    P.vx = static_cast<float>(c->vox[0]); P.vy = static_cast<float>(c->vox[1]); P.vz = static_cast<float>(c->vox[2]);
    P.ivx = 1.0f / P.vx; P.ivy = 1.0f / P.vy; P.ivz = 1.0f / P.vz;
    P.rho = c->d_rho;
    P.rho_hom = c->d_rho_hom;
    for (int m = 0; m < 4; ++m) P.rho_max[m] = c->rho_max[m];
    P.mgM = c->mgM; P.mgx = c->mg[0]; P.mgy = c->mg[1]; P.mgz = c->mg[2];
    P.mgrid = c->d_mgrid;
    for (int k = 0; k < 3; ++k) P.thr[k] = c->thr[k];
    P.fields = c->d_fields;
    P.n_fields = nfields(c);
    P.first = c->d_first;
    const mc_epid_desc& E = c->epid;
    P.nl = E.n_layers; P.sens = E.sensitive_layer; P.npx = E.npx; P.npy = E.npy;
    P.pitch = static_cast<float>(E.pitch_cm);
    P.ipitch = 1.0f / P.pitch;
    P.hwx = static_cast<float>(0.5 * E.npx * E.pitch_cm);
    P.hwy = static_cast<float>(0.5 * E.npy * E.pitch_cm);
    for (int l = 0; l <= E.n_layers; ++l) P.zp[l] = static_cast<float>(c->zp[l] - c->zp[0]);
    for (int l = 0; l < E.n_layers; ++l) {
        P.lmat[l] = E.material[l];
        P.lrho[l] = static_cast<float>(E.density[l]);
    }
    P.rect = c->d_rect; P.cdf = c->d_cdf; P.guide = c->d_guide; P.rflag = c->d_rflag;
    {
        const mcphys::MaterialCoefs w = mcphys::tungsten_coefs();
        P.wmat = {static_cast<float>(w.ne_barn), static_cast<float>(w.pe_above), static_cast<float>(w.pe_below),
                  static_cast<float>(w.pair), 0.0f, 0.0f};
        P.w_edge = static_cast<float>(mcphys::kWKEdge);
    }
    P.e_max = static_cast<float>(c->cfg.e_max_mev);
    P.mono_e = static_cast<float>(c->cfg.mono_energy_mev);
    P.pcut = static_cast<float>(c->cfg.photon_cutoff_mev);
    P.ecut = static_cast<float>(c->cfg.electron_cutoff_mev);
    P.tstop = P.ecut + mc::kStopMargin;
    P.wcc = static_cast<float>(c->cfg.wcc_mev);
    P.wcb = static_cast<float>(c->cfg.wcb_mev);
    P.ln_wcb = logf(P.wcb);
    P.step_frac = static_cast<float>(c->cfg.step_fraction);
    P.max_steps = c->cfg.max_steps;
    P.coupled = c->cfg.coupled;
    P.nbatch = c->cfg.n_batches;
    for (int m = 0; m < mc::kNumMat; ++m) {
        const mcphys::MaterialCoefs& k = c->tabs.mat[m];
        P.mat[m] = {static_cast<float>(k.ne_barn), static_cast<float>(k.pe_above), static_cast<float>(k.pe_below),
                    static_cast<float>(k.pair), static_cast<float>(k.brem), static_cast<float>(k.msc)};
    }
    P.ptab = c->d_ptab;
    P.p_lnE0 = static_cast<float>(c->tabs.p_lnE0);
    P.p_idx = static_cast<float>(c->tabs.p_inv_dlnE);
    P.etab = c->d_etab;
    P.e_lnT0 = static_cast<float>(c->tabs.e_lnT0);
    P.e_idx = static_cast<float>(c->tabs.e_inv_dlnT);
    P.w_lnG0 = static_cast<float>(c->tabs.w_lnG0);
    P.w_idx = static_cast<float>(c->tabs.w_inv_dlnG);
    P.seed = seed;
    P.key = mc::philox_key(seed);
    P.tally = c->d_tally;
    P.energy = c->d_energy;
    P.events = c->d_events;
    P.vox = c->cfg.patient_dose ? c->d_vox : nullptr;
    P.ctl = c->d_ctl;
    P.heads = c->d_heads;
    for (int t = 0; t < mc::kNumBanks; ++t)
        for (int k = 0; k < 2; ++k) P.bank[t][k] = c->bank[t][k];
    P.cap = c->cap;
    P.flush_lanes = 8;
    // CT-photon slot pools: at most 1/16 of a bank can be left reserved but
    // unused at the end of a launch (16 slots per warp for the benchmark's
    // banks; 16 measured slightly better than 32)
    {
        const unsigned long long warps =
            static_cast<unsigned long long>(c->grid[mc::kPhotonCT]) * static_cast<unsigned long long>(c->block) / 32u;
        const unsigned long long per = warps ? static_cast<unsigned long long>(c->cap) / (16u * warps) : 1u;
        P.pool_chunk = static_cast<uint32_t>(std::max<unsigned long long>(1u, std::min<unsigned long long>(16u, per)));
    }
}

bool increasing(const double* a, int n) {
    for (int i = 1; i < n; ++i)
        if (!(a[i] > a[i - 1])) return false;
    return true;
}

// Source rectangles of one field (weight MU x open area, cumulative in
// double, appended to rect / cdf), its bounding box, Eq. 1 and beam frame.
mc_status build_field(mc_ctx* c, const mc_field_desc* f, int index, std::vector<float4>& rect,
                      std::vector<double>& cdf, std::vector<unsigned char>& rflag, FieldHost& out) {
    const std::string which = " (field " + std::to_string(index) + ")";
    if (!f->pair_edges_cm || !f->leaves_cm || !f->jaws_cm || !f->mu) return fail(c, MC_ERR_ARG, "null field" + which);
    if (f->n_segments < 1 || f->n_pairs < 1 || f->n_segments * f->n_pairs > (1 << 20))
        return fail(c, MC_ERR_ARG, "bad segment / pair count" + which);
    if (!(f->sad_cm > 0) || !(f->sid_cm > f->sad_cm)) return fail(c, MC_ERR_ARG, "need 0 < SAD < SID" + which);
    if (!increasing(f->pair_edges_cm, f->n_pairs + 1)) return fail(c, MC_ERR_ARG, "pair edges must increase" + which);
    const double T = f->leaf_transmission, Tj = f->jaw_transmission;
    const double w = f->tg_width_cm, gap = f->leaf_gap_cm;
    if (!(T >= 0.0 && T < 1.0) || !(Tj >= 0.0 && Tj < 1.0))
        return fail(c, MC_ERR_ARG, "leaf and jaw transmission must be in [0, 1)" + which);
    double narrowest = INFINITY;
    for (int j = 0; j < f->n_pairs; ++j)
        narrowest = std::fmin(narrowest, f->pair_edges_cm[j + 1] - f->pair_edges_cm[j]);
    if (!(w >= 0.0 && w < narrowest)) return fail(c, MC_ERR_ARG, "tongue-and-groove width must be in [0, narrowest pair)" + which);
    if (!(gap >= 0.0 && gap < 2.0)) return fail(c, MC_ERR_ARG, "leaf gap must be in [0, 2) cm" + which);
    const double tl = f->leaf_thickness_cm, tj = f->jaw_thickness_cm;
    if (!(tl >= 0.0 && tl <= 20.0) || !(tj >= 0.0 && tj < 23.0))
        return fail(c, MC_ERR_ARG, "need 0 <= leaf slab <= 20 cm and 0 <= jaw slab < 23 cm" + which);
    // collimator slabs: every rectangle weighs MU x area and carries the slabs
    // its photons cross; they replace the transmission factors
    const bool slab = tl > 0.0 || tj > 0.0;
    if (slab && (T > 0.0 || Tj > 0.0))
        return fail(c, MC_ERR_ARG, "collimator slabs replace the transmission factors: set those to 0" + which);
    const size_t off = rect.size();
    double acc = 0.0, X0 = INFINITY, X1 = -INFINITY, Y0 = INFINITY, Y1 = -INFINITY;
    bool open = false;
    auto add = [&](double x0, double x1, double y0, double y1, double wt, unsigned char flag) {
        if (!(x1 > x0) || !(y1 > y0) || !(wt > 0.0)) return;
        acc += wt * (x1 - x0) * (y1 - y0);
        rect.push_back(make_float4(static_cast<float>(x0), static_cast<float>(x1), static_cast<float>(y0),
                                   static_cast<float>(y1)));
        rflag.push_back(flag);
        cdf.push_back(acc);
    };
    // [lo, hi] framed and split at the cuts strictly inside it, ascending, distinct
    auto split = [](double lo, double hi, std::initializer_list<double> cuts) {
        std::vector<double> v{lo};
        for (double x : cuts)
            if (x > lo && x < hi) v.push_back(x);
        std::sort(v.begin() + 1, v.end());
        v.push_back(hi);
        v.erase(std::unique(v.begin(), v.end()), v.end());
        return v;
    };
    constexpr double kHalf = 20.0;            // the largest field, 40 x 40 cm at the isocentre
    // Every (segment, pair, Y band, X interval) on which the leaf and jaw
    // factors are constant is one source rectangle of weight MU x factors,
    // in that order; the same order as the oracle, so replay keys match.
    for (int k = 0; k < f->n_segments; ++k) {
        const double* jw = f->jaws_cm + 4 * k;
        const double mu = f->mu[k];
        if (!(mu >= 0.0)) return fail(c, MC_ERR_ARG, "MU weights must be >= 0" + which);
        if (!(mu > 0.0)) continue;
        const double jx0 = std::fmax(jw[0], -kHalf), jx1 = std::fmin(jw[1], kHalf);
        const double jy0 = std::fmax(jw[2], -kHalf), jy1 = std::fmin(jw[3], kHalf);
        const double* lv = f->leaves_cm + 2 * static_cast<size_t>(k) * f->n_pairs;
        // effective opening of pair j: tips apart by the leaf gap, if open at all
        auto opening = [&](int j, double& lo, double& hi) {
            if (!(lv[2 * j + 1] > lv[2 * j])) return false;
            lo = lv[2 * j] - 0.5 * gap;
            hi = lv[2 * j + 1] + 0.5 * gap;
            return true;
        };
        for (int j = 0; j < f->n_pairs; ++j) {
            const double e0 = f->pair_edges_cm[j], e1 = f->pair_edges_cm[j + 1];
            // the physical aperture sets the field size of Eq. 1
            const double ax0 = std::fmax(lv[2 * j], jw[0]), ax1 = std::fmin(lv[2 * j + 1], jw[1]);
            const double ay0 = std::fmax(e0, jw[2]), ay1 = std::fmin(e1, jw[3]);
            if (ax1 > ax0 && ay1 > ay0) {
                open = true;
                X0 = std::fmin(X0, ax0); X1 = std::fmax(X1, ax1); Y0 = std::fmin(Y0, ay0); Y1 = std::fmax(Y1, ay1);
            }
            const double ya = std::fmax(e0, -kHalf), yb = std::fmin(e1, kHalf);
            if (!(yb > ya)) continue;
            const std::vector<double> ys = w > 0.0 ? split(ya, yb, {jy0, jy1, e0 + 0.5 * w, e1 - 0.5 * w})
                                                   : split(ya, yb, {jy0, jy1});
            for (size_t b = 0; b + 1 < ys.size(); ++b) {
                const double y0 = ys[b], y1 = ys[b + 1], ym = 0.5 * (y0 + y1);
                double lo = 0.0, hi = 0.0;
                bool has = opening(j, lo, hi);
                int nb = -1;                      // pair sharing this tongue-and-groove strip
                if (w > 0.0 && j > 0 && ym < e0 + 0.5 * w) nb = j - 1;
                if (w > 0.0 && j + 1 < f->n_pairs && ym > e1 - 0.5 * w) nb = j + 1;
                if (has && nb >= 0) {
                    double lo2, hi2;
                    has = opening(nb, lo2, hi2);
                    if (has) {
                        lo = std::fmax(lo, lo2);
                        hi = std::fmin(hi, hi2);
                        has = hi > lo;
                    }
                }
                const bool jaw_y = ym >= jy0 && ym <= jy1;
                const std::vector<double> xs = has ? split(-kHalf, kHalf, {jx0, jx1, lo, hi})
                                                   : split(-kHalf, kHalf, {jx0, jx1});
                for (size_t a2 = 0; a2 + 1 < xs.size(); ++a2) {
                    const double x0 = xs[a2], x1 = xs[a2 + 1], xm = 0.5 * (x0 + x1);
                    const bool in_leaf = has && xm >= lo && xm <= hi;
                    const bool in_jaw = jaw_y && xm >= jx0 && xm <= jx1;
                    const double leaf = in_leaf ? 1.0 : (slab ? (tl > 0.0 ? 1.0 : 0.0) : T);
                    const double jaw = in_jaw ? 1.0 : (slab ? (tj > 0.0 ? 1.0 : 0.0) : Tj);
                    const unsigned char flag = slab ? static_cast<unsigned char>((in_leaf ? 0 : 1) | (in_jaw ? 0 : 2)) : 0;
                    add(x0, x1, y0, y1, mu * leaf * jaw, flag);
                }
            }
        }
    }
    if (!(acc > 0.0)) open = false;
    if (!open) return fail(c, MC_ERR_ARG, "field has no open aperture" + which);
    for (size_t i = off; i < cdf.size(); ++i) cdf[i] /= acc;
    out.rect_off = static_cast<int>(off);
    out.n_rect = static_cast<int>(rect.size() - off);
    out.bbox_a = X1 - X0;
    out.bbox_b = Y1 - Y0;
    // Eq. 1 as printed gives ab / (2(a+b)) (2.5 cm for 10 x 10), which cannot index
    // Table 1; the default reading is the equivalent square 2ab / (a+b).
    out.s_eq = f->eq1_literal ? out.bbox_a * out.bbox_b / (2.0 * (out.bbox_a + out.bbox_b))
                              : 2.0 * out.bbox_a * out.bbox_b / (out.bbox_a + out.bbox_b);
    const double g = f->gantry_deg * 3.14159265358979323846 / 180.0;
    out.ex[0] = std::cos(g); out.ex[1] = std::sin(g); out.ex[2] = 0.0;
    out.ey[0] = 0.0; out.ey[1] = 0.0; out.ey[2] = 1.0;
    out.ez[0] = std::sin(g); out.ez[1] = -std::cos(g); out.ez[2] = 0.0;
    for (int k = 0; k < 3; ++k) out.iso[k] = f->iso_cm[k];
    out.sad = f->sad_cm;
    out.sid = f->sid_cm;
    out.leaf_t = tl;
    out.jaw_t = tj;
    out.zface = (out.sad - out.sid) + c->zp[0];
    // the vacuum transfer needs the whole CT above the detector face and below the source
    for (int corner = 0; corner < 8; ++corner) {
        double p[3];
        const int n[3] = {c->nx, c->ny, c->nz};
        for (int k = 0; k < 3; ++k) p[k] = c->origin[k] + ((corner >> k) & 1) * n[k] * c->vox[k] - out.iso[k];
        const double Z = p[0] * out.ez[0] + p[1] * out.ez[1] + p[2] * out.ez[2];
        if (!(Z > out.zface + 1e-3) || !(Z < out.sad))
            return fail(c, MC_ERR_ARG, "CT box must lie between the source and the EPID face" + which);
    }
    out.stream_base = static_cast<uint64_t>(index) * kFieldStride;
    out.hist_done = 0;
    return MC_OK;
}

// Per-field device records for a run; `first` is the prefix sum of the
// histories each field runs in it.
mc_status upload_fields(mc_ctx* c, const std::vector<uint64_t>& first, cudaStream_t s) {
    // pinned staging: the previous run (whose copies read it) has finished
    FieldDev* fd = c->h_fields;
    const size_t per_field = static_cast<size_t>(c->cfg.n_batches) * npix(c);
    for (size_t i = 0; i < c->fields.size(); ++i) {
        const FieldHost& h = c->fields[i];
        FieldDev& d = fd[i];
        for (int k = 0; k < 3; ++k) {
            d.ex[k] = static_cast<float>(h.ex[k]);
            d.ey[k] = static_cast<float>(h.ey[k]);
            d.ez[k] = static_cast<float>(h.ez[k]);
            d.iso[k] = static_cast<float>(h.iso[k]);
        }
        d.sad = static_cast<float>(h.sad);
        d.zface = static_cast<float>(h.zface);
        d.leaf_t = static_cast<float>(h.leaf_t);
        d.jaw_t = static_cast<float>(h.jaw_t);
        d.rect_off = h.rect_off;
        d.n_rect = h.n_rect;
        d.hist_base = h.stream_base + h.hist_done;
        d.batch_base = h.hist_done;
        d.tally_off = i * per_field;
    }
    for (size_t i = 0; i < first.size(); ++i) c->h_first[i] = first[i];
    CUDA_TRY(c, cudaMemcpyAsync(c->d_fields, fd, sizeof(FieldDev) * c->fields.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_first, c->h_first, sizeof(unsigned long long) * first.size(),
                                cudaMemcpyHostToDevice, s));
    return MC_OK;
}

struct WaveResult {
    int waves = 0;
    uint32_t launches = 0;
    uint32_t klaunch[4] = {0, 0, 0, 0};
    double kms[4] = {0, 0, 0, 0};
};


const int kOrder[4] = {mc::kPhotonCT, mc::kElectronCT, mc::kPhotonEPID, mc::kElectronEPID};

// Graph-driven waves: one wave (wave-begin, the transport kernels with their
// bank swaps, wave-end) is captured into the body of a conditional while-node;
// the wave-end kernel sets the condition, so the whole run is one launch and
// the host waits once.  `e0` is recorded just before the launch.
mc_status run_waves_graph(mc_ctx* c, const Params& P, cudaStream_t s, WaveResult& r) {
    if (!c->capture_stream) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    };
    CUDA_TRY(c, cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np{};
    cudaGraphNode_t node;
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = handle;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    }
    if (e != cudaSuccess) {
        cleanup();
        return fail(c, MC_ERR_CUDA, std::string("conditional node: ") + cudaGetErrorString(e));
    }
    cudaStream_t cs = c->capture_stream;
    e = cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cleanup();
        return fail(c, MC_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    }
    uint32_t per_wave = 3;   // wave-begin, source and wave-end
    e = mc::launch_wave_begin(c->d_ctl, c->cfg.primaries_per_wave, c->cfg.bank_capacity, cs);
    if (e == cudaSuccess) e = mc::launch_source(P, c->src_grid, cs);
    for (int t : kOrder) {
        if (is_electron(t) && !c->cfg.coupled) continue;
        if (e == cudaSuccess) e = mc::launch_transport(t, c->minb[t], P, c->grid[t], c->block, cs);
        if (e == cudaSuccess) e = mc::launch_swap(c->d_ctl, c->d_heads, t, c->cap, cs);
        per_wave += 2;
    }
    if (e == cudaSuccess) e = mc::launch_wave_end(c->d_ctl, handle, kMaxWaves, cs);
    cudaGraph_t captured = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(cs, &captured);
    if (e == cudaSuccess) e = e_end;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_run0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    // the control block comes back with the run; the host reads it (and the
    // events) only when asked (finalize_run), so the call does not wait
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_run1, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);    // a launched graph must finish before it is destroyed
        cleanup();
        return fail(c, MC_ERR_CUDA, std::string("graph-driven run: ") + cudaGetErrorString(e));
    }
    // the graph stays alive until finalize_run (destroying it here would wait)
    c->run_graph = graph;
    c->run_exec = exec;
    c->run_pending = true;
    c->run_per_wave = per_wave;
    r.waves = -1;
    return MC_OK;
}

// Host-driven waves: the host reads the run control after every wave and
// stops when all banks are empty; it can time every transport launch.
mc_status run_waves_host(mc_ctx* c, const Params& P, cudaStream_t s, cudaEvent_t e0, WaveResult& r) {
    Ctl& h = *c->h_ctl;
    std::vector<std::pair<int, size_t>> timed;   // (type, index of its start event)
    size_t ev_used = 0;
    auto next_event = [&]() -> cudaEvent_t {
        if (ev_used == c->ev_pool.size()) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            c->ev_pool.push_back(ev);
        }
        return c->ev_pool[ev_used++];
    };
    CUDA_TRY(c, cudaEventRecord(e0, s));
    mc_status result = MC_OK;
    int& waves = r.waves;
    for (; waves < static_cast<int>(kMaxWaves); ++waves) {
        CUDA_TRY(c, mc::launch_wave_begin(c->d_ctl, c->cfg.primaries_per_wave, c->cfg.bank_capacity, s));
        CUDA_TRY(c, mc::launch_source(P, c->src_grid, s));
        r.launches += 2;
        for (int t : kOrder) {
            if (is_electron(t) && !c->cfg.coupled) continue;
            if (c->cfg.time_kernels) {
                timed.emplace_back(t, ev_used);
                CUDA_TRY(c, cudaEventRecord(next_event(), s));
            }
            CUDA_TRY(c, mc::launch_transport(t, c->minb[t], P, c->grid[t], c->block, s));
            if (c->cfg.time_kernels) CUDA_TRY(c, cudaEventRecord(next_event(), s));
            CUDA_TRY(c, mc::launch_swap(c->d_ctl, c->d_heads, t, c->cap, s));
            r.launches += 2;
            ++r.klaunch[t];
        }
        CUDA_TRY(c, cudaMemcpyAsync(&h, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (h.error) { result = fail(c, MC_ERR_OVERFLOW, "particle bank overflow"); ++waves; break; }
        bool empty = h.next_prim >= h.n_total;
        for (int t = 0; t < mc::kNumBanks; ++t) empty = empty && h.count[t][h.cur[t]] == 0u;
        if (empty) { ++waves; break; }
        if (c->cancel.load()) { result = fail(c, MC_ERR_CANCELLED, "cancelled"); ++waves; break; }
    }
    if (waves >= static_cast<int>(kMaxWaves) && result == MC_OK) result = fail(c, MC_ERR_TIMEOUT, "wave limit reached");
    for (const auto& te : timed) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev_pool[te.second], c->ev_pool[te.second + 1]);
        r.kms[te.first] += ms;
    }
    return result;
}

mc_status set_fields_impl(mc_ctx* c, const mc_field_desc* f, int n, const mc_lut_desc* lut, cudaStream_t s) {
    if (!c->has_geom) return fail(c, MC_ERR_STATE, "mc_init_geometry must come first");
    if (!f || n < 1 || n > mc::kMaxFields) return fail(c, MC_ERR_ARG, "need 1..256 fields");
    if (lut) {
        if (lut->nt < 2 || lut->ns < 2 || lut->nt > 1024 || lut->ns > 1024 || !lut->t_nodes || !lut->s_nodes || !lut->k)
            return fail(c, MC_ERR_ARG, "bad k-table");
        if (!increasing(lut->t_nodes, lut->nt) || !increasing(lut->s_nodes, lut->ns))
            return fail(c, MC_ERR_ARG, "k-table nodes must increase");
    }
    CUDA_TRY(c, cudaSetDevice(c->device));
    std::vector<float4> rect;
    std::vector<double> cdf;
    std::vector<unsigned char> rflag;
    std::vector<FieldHost> fh(n);
    for (int i = 0; i < n; ++i) {
        const mc_status st = build_field(c, &f[i], i, rect, cdf, rflag, fh[i]);
        if (st != MC_OK) return st;
    }
    const int np = npix(c);
    const size_t tally_n = static_cast<size_t>(n) * c->cfg.n_batches * np;
    const size_t parts = (np + 255) / 256;
    const size_t nks = lut ? static_cast<size_t>(n) * lut->nt : 0;
    // Buffers are kept while large enough, and then nothing here waits for
    // the device.  A buffer that must grow is replaced, which needs the
    // previous run to have finished with it.
    const bool grow = tally_n > c->cap_tally || static_cast<size_t>(np) > c->cap_pix || parts > c->cap_parts ||
                      rect.size() > c->cap_rect || cdf.size() > c->cap_cdf || rflag.size() > c->cap_rflag ||
                      rect.size() > c->cap_guide ||
                      static_cast<size_t>(n) * np > c->cap_tmap || (lut && (static_cast<size_t>(lut->nt) > c->cap_lut_t ||
                                                                             nks > c->cap_ks));
    if (grow) {
        const mc_status prev = finalize_run(c);
        if (prev != MC_OK) return prev;
    } else {
        const mc_status o = order_after_run(c, s);
        if (o != MC_OK) return o;
    }
    clear_fields(c);
    CUDA_TRY(c, ensure(c->d_tally, c->cap_tally, tally_n));
    c->tally_n = tally_n;
    size_t cp = c->cap_pix;
    CUDA_TRY(c, ensure(c->d_dose, cp, static_cast<size_t>(np)));
    cp = c->cap_pix;
    CUDA_TRY(c, ensure(c->d_sigma, cp, static_cast<size_t>(np)));
    cp = c->cap_pix;
    CUDA_TRY(c, ensure(c->d_signal, cp, static_cast<size_t>(np)));
    cp = c->cap_pix;
    CUDA_TRY(c, ensure(c->d_flu, cp, static_cast<size_t>(np)));
    c->cap_pix = cp;
    size_t cq = c->cap_parts;
    CUDA_TRY(c, ensure(c->d_part, cq, parts));
    cq = c->cap_parts;
    CUDA_TRY(c, ensure(c->d_partc, cq, parts));
    c->cap_parts = cq;
    CUDA_TRY(c, ensure(c->d_rect, c->cap_rect, rect.size()));
    CUDA_TRY(c, ensure(c->d_cdf, c->cap_cdf, cdf.size()));
    CUDA_TRY(c, ensure(c->d_rflag, c->cap_rflag, rflag.size()));
    CUDA_TRY(c, ensure(c->d_guide, c->cap_guide, rect.size()));
    CUDA_TRY(c, ensure(c->d_tmap, c->cap_tmap, static_cast<size_t>(n) * np));
    // host data to the device through pinned staging, so the copies need no
    // wait here; the staging is reused once the previous copies out of it ended
    // cut points of every field's CDF: the source search starts at
    // guide[floor(xi n)] and scans to the first rectangle whose cumulative
    // weight exceeds xi, the same rectangle a binary search finds
    std::vector<uint32_t> guide(rect.size());
    for (int i = 0; i < n; ++i) {
        const int off = fh[i].rect_off, nr = fh[i].n_rect;
        int r = 0;
        for (int j = 0; j < nr; ++j) {
            const double u = static_cast<double>(j) / nr;
            while (r < nr - 1 && u >= cdf[off + r]) ++r;
            guide[off + j] = static_cast<uint32_t>(r);
        }
    }
    const size_t stage_bytes = sizeof(float4) * rect.size() + sizeof(double) * (cdf.size() + nks + (lut ? lut->nt : 0)) +
                               sizeof(uint32_t) * guide.size() + rflag.size();
    CUDA_TRY(c, cudaEventSynchronize(c->ev_stage));
    if (stage_bytes > c->h_stage_cap) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_cap = 0;
        CUDA_TRY(c, cudaMallocHost(&c->h_stage, stage_bytes));
        c->h_stage_cap = stage_bytes;
    }
    char* stage = c->h_stage;
    float4* h_rect = reinterpret_cast<float4*>(stage);
    double* h_cdf = reinterpret_cast<double*>(stage + sizeof(float4) * rect.size());
    double* h_ks = h_cdf + cdf.size();
    double* h_lut_t = h_ks + nks;
    uint32_t* h_guide = reinterpret_cast<uint32_t*>(h_lut_t + (lut ? lut->nt : 0));
    unsigned char* h_rflag = reinterpret_cast<unsigned char*>(h_guide + guide.size());
    std::memcpy(h_guide, guide.data(), sizeof(uint32_t) * guide.size());
    CUDA_TRY(c, cudaMemcpyAsync(c->d_guide, h_guide, sizeof(uint32_t) * guide.size(), cudaMemcpyHostToDevice, s));
    std::memcpy(h_rect, rect.data(), sizeof(float4) * rect.size());
    std::memcpy(h_cdf, cdf.data(), sizeof(double) * cdf.size());
    std::memcpy(h_rflag, rflag.data(), rflag.size());
    CUDA_TRY(c, cudaMemcpyAsync(c->d_rflag, h_rflag, rflag.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_rect, h_rect, sizeof(float4) * rect.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_cdf, h_cdf, sizeof(double) * cdf.size(), cudaMemcpyHostToDevice, s));

    // radiological thickness map of every field (Sec. 2.2)
    c->t_offset = lut ? lut->t_offset_cm : 0.0;
    const mc_epid_desc& E = c->epid;
    for (int i = 0; i < n; ++i) {
        const FieldHost& h = fh[i];
        mc::TmapArgs A;
        A.nx = c->nx; A.ny = c->ny; A.nz = c->nz;
        A.ox = static_cast<float>(c->origin[0]); A.oy = static_cast<float>(c->origin[1]);
        A.oz = static_cast<float>(c->origin[2]);
        A.vx = static_cast<float>(c->vox[0]); A.vy = static_cast<float>(c->vox[1]);
        A.vz = static_cast<float>(c->vox[2]);
        A.rho = c->d_rho;
        for (int k = 0; k < 3; ++k) {
            A.src[k] = static_cast<float>(h.iso[k] + h.sad * h.ez[k]);
            A.iso[k] = static_cast<float>(h.iso[k]);
            A.ex[k] = static_cast<float>(h.ex[k]);
            A.ey[k] = static_cast<float>(h.ey[k]);
            A.ez[k] = static_cast<float>(h.ez[k]);
        }
        A.npx = E.npx; A.npy = E.npy;
        A.pitch = static_cast<float>(E.pitch_cm);
        A.hwx = static_cast<float>(0.5 * E.npx * E.pitch_cm);
        A.hwy = static_cast<float>(0.5 * E.npy * E.pitch_cm);
        A.zs = static_cast<float>(h.sad - h.sid);
        A.t_offset = c->t_offset;
        CUDA_TRY(c, mc::launch_tmap(A, c->d_tmap + static_cast<size_t>(i) * np, s));
    }

    // k-table: the column at each field's s, for the per-pixel step along t
    if (lut) {
        for (int i = 0; i < n; ++i) {
            const double sc = std::fmin(std::fmax(fh[i].s_eq, lut->s_nodes[0]), lut->s_nodes[lut->ns - 1]);
            int js = 0;
            while (js + 1 < lut->ns - 1 && lut->s_nodes[js + 1] <= sc) ++js;
            const double fs = (sc - lut->s_nodes[js]) / (lut->s_nodes[js + 1] - lut->s_nodes[js]);
            for (int it = 0; it < lut->nt; ++it)
                h_ks[static_cast<size_t>(i) * lut->nt + it] = (1.0 - fs) * lut->k[static_cast<size_t>(js) * lut->nt + it] +
                                                               fs * lut->k[static_cast<size_t>(js + 1) * lut->nt + it];
        }
        std::memcpy(h_lut_t, lut->t_nodes, sizeof(double) * lut->nt);
        CUDA_TRY(c, ensure(c->d_lut_t, c->cap_lut_t, static_cast<size_t>(lut->nt)));
        CUDA_TRY(c, ensure(c->d_lut_ks, c->cap_ks, nks));
        CUDA_TRY(c, cudaMemcpyAsync(c->d_lut_t, h_lut_t, sizeof(double) * lut->nt, cudaMemcpyHostToDevice, s));
        CUDA_TRY(c, cudaMemcpyAsync(c->d_lut_ks, h_ks, sizeof(double) * nks, cudaMemcpyHostToDevice, s));
        c->lut_nt = lut->nt;
        c->k_scale = lut->k_scale;
        c->has_lut = true;
    }
    CUDA_TRY(c, cudaEventRecord(c->ev_stage, s));
    c->fields = fh;
    const mc_status st = clear_tally(c, s);
    if (st != MC_OK) return st;
    c->has_field = true;
    return MC_OK;
}

mc_status run_impl(mc_ctx* c, const uint64_t* n, uint64_t seed, cudaStream_t s, mc_run_stats* stats) {
    if (!c->has_field) return fail(c, MC_ERR_STATE, "mc_set_field must come first");
    std::vector<uint64_t> first(c->fields.size() + 1, 0);
    for (size_t i = 0; i < c->fields.size(); ++i) {
        if (n[i] > 0xffffffffull) return fail(c, MC_ERR_ARG, "at most 2^32-1 histories per field and call");
        first[i + 1] = first[i] + n[i];
    }
    CUDA_TRY(c, cudaSetDevice(c->device));
    // a previous graph-driven run still in flight: wait for it (its control
    // block and the pinned staging are reused) and report its outcome
    const mc_status prev = finalize_run(c);
    if (prev != MC_OK) return prev;
    c->cancel.store(0);
    mc_status st = upload_fields(c, first, s);
    if (st != MC_OK) return st;
    Params P;
    make_params(c, P, seed);
    Ctl& h = *c->h_ctl;
    std::memset(&h, 0, sizeof(h));
    h.n_total = first.back();
    CUDA_TRY(c, cudaMemcpyAsync(c->d_ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemsetAsync(c->d_heads, 0, kHeadsBytes, s));
    for (size_t i = 0; i < c->fields.size(); ++i) c->fields[i].hist_done += n[i];
    WaveResult r;
    // per-kernel timing needs the host-driven loop
    if (c->cfg.use_graph && !c->cfg.time_kernels) {
        const mc_status result = run_waves_graph(c, P, s, r);
        if (result != MC_OK) return result;
        if (!stats) return MC_OK;                 // queued on s; nothing waited for
        const mc_status outcome = finalize_run(c);
        const mc_status s2 = mc_get_stats(c, stats);
        return outcome != MC_OK ? outcome : s2;
    }
    const mc_status result = run_waves_host(c, P, s, c->ev_run0, r);
    float ms = 0.f;
    if (cudaEventRecord(c->ev_run1, s) == cudaSuccess && cudaEventSynchronize(c->ev_run1) == cudaSuccess)
        cudaEventElapsedTime(&ms, c->ev_run0, c->ev_run1);
    c->last_waves = r.waves;
    c->last_error = h.error;
    c->last_ms = ms;
    c->last_launches = r.launches;
    for (int t = 0; t < 4; ++t) { c->last_kernel_ms[t] = r.kms[t]; c->last_kernel_launches[t] = r.klaunch[t]; }
    if (stats) {
        const mc_status s2 = mc_get_stats(c, stats);
        if (s2 != MC_OK) return s2;
    }
    return result;
}

mc_status compute_dose(mc_ctx* c, int field, double* dose, double* sigma, double* u_dev, cudaStream_t s) {
    const int B = c->cfg.n_batches;
    const uint64_t N = c->fields[field].hist_done;
    if (N == 0) return fail(c, MC_ERR_STATE, "no histories run");
    CUDA_TRY(c, mc::launch_batch_counts(c->d_nb, B, N, s));
    const mc_epid_desc& E = c->epid;
    const int l = E.sensitive_layer;
    const double mass_kg = E.density[l] * E.pitch_cm * E.pitch_cm * E.thickness_cm[l] * 1e-3;
    const unsigned long long* tally = c->d_tally + static_cast<size_t>(field) * B * npix(c);
    CUDA_TRY(c, mc::launch_dose(tally, npix(c), B, c->d_nb, static_cast<double>(N), kJoulePerMeV / mass_kg, dose,
                                sigma, c->d_maxbits, c->d_part, c->d_partc, u_dev, s));
    return MC_OK;
}

mc_status check_field(mc_ctx* c, int field) {
    if (!c->has_field) return fail(c, MC_ERR_STATE, "no field");
    if (field < 0 || field >= nfields(c)) return fail(c, MC_ERR_ARG, "field index out of range");
    return MC_OK;
}

// State layout (uint64 words): magic, B, npx, npy, number of fields, voxels
// of the patient-dose tally (0 when off), the next history index of each
// field, energy counters, event counters, sub-tallies, patient-dose tally.
const uint64_t kStateMagic = 0x4550494453543033ull;   // "EPIDST03"
constexpr size_t kStateHead = 6;
size_t vox_words(const mc_ctx* c) { return c->cfg.patient_dose ? c->vox_n : 0; }
size_t state_words(const mc_ctx* c) {
    return kStateHead + c->fields.size() + mc::kNumEnergy + mc::kNumEvents + c->tally_n + vox_words(c);
}

}  // namespace

extern "C" {

void mc_config_default(mc_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->coupled = 1;
    cfg->e_max_mev = 6.0;
    cfg->mono_energy_mev = 0.0;
    cfg->photon_cutoff_mev = 0.01;
    cfg->electron_cutoff_mev = 0.2;
    cfg->wcc_mev = 0.2;
    cfg->wcb_mev = 0.01;
    cfg->step_fraction = 0.05;
    cfg->n_batches = 16;
    cfg->max_steps = 10000;
    cfg->block_size = 256;
    cfg->ctas_per_sm = 0;
    cfg->bank_capacity = 1u << 23;
    cfg->primaries_per_wave = 0;
    cfg->time_kernels = 0;
    cfg->use_graph = 1;
    for (int t = 0; t < 4; ++t) cfg->regs_variant[t] = kDefaultRegsVariant[t];
    cfg->patient_dose = 0;
}

const char* mc_status_string(mc_status s) {
    switch (s) {
        case MC_OK: return "ok";
        case MC_ERR_ARG: return "invalid argument";
        case MC_ERR_CUDA: return "CUDA error";
        case MC_ERR_OOM: return "out of device memory";
        case MC_ERR_STATE: return "call out of order";
        case MC_ERR_TIMEOUT: return "bounded wait exceeded";
        case MC_ERR_CANCELLED: return "cancelled";
        case MC_ERR_NUMERIC: return "non-finite value";
        case MC_ERR_OVERFLOW: return "particle bank overflow";
    }
    return "unknown status";
}

const char* mc_last_error(const mc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mc_status mc_create(const mc_config* cfg_in, int device, mc_ctx** out) {
    if (!out) return MC_ERR_ARG;
    *out = nullptr;
    mc_config cfg;
    if (cfg_in) cfg = *cfg_in; else mc_config_default(&cfg);
    if (cfg.block_size == 0) cfg.block_size = 256;
    if (cfg.bank_capacity == 0) cfg.bank_capacity = 1u << 23;
    for (int t = 0; t < 4; ++t) {
        if (cfg.regs_variant[t] == 0) cfg.regs_variant[t] = kDefaultRegsVariant[t];
        if (cfg.regs_variant[t] < 2 || cfg.regs_variant[t] > 4) return MC_ERR_ARG;
    }
    if (cfg.primaries_per_wave == 0) cfg.primaries_per_wave = cfg.bank_capacity / 4;
    if (cfg.block_size % 32 != 0 || cfg.block_size < 32 || cfg.block_size > 256) return MC_ERR_ARG;
    if (cfg.n_batches < 2 || cfg.n_batches > 1024 || cfg.max_steps < 1) return MC_ERR_ARG;
    if (!(cfg.photon_cutoff_mev > 0) || !(cfg.electron_cutoff_mev > 0) || !(cfg.wcb_mev > 0) ||
        !(cfg.wcc_mev > 0) || !(cfg.step_fraction > 0 && cfg.step_fraction < 1) || !(cfg.e_max_mev > 0))
        return MC_ERR_ARG;
    if (cfg.bank_capacity < 1024 || cfg.primaries_per_wave < 32) return MC_ERR_ARG;
    if (cfg.use_graph != 0 && cfg.use_graph != 1) return MC_ERR_ARG;
    if (cfg.patient_dose != 0 && cfg.patient_dose != 1) return MC_ERR_ARG;

    mc_ctx* c = new mc_ctx();
    c->cfg = cfg;
    c->device = device;
    auto bail = [&](mc_status s) { mc_destroy(c); return s; };
    if (cudaSetDevice(device) != cudaSuccess) return bail(MC_ERR_CUDA);
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bail(MC_ERR_CUDA);

    const double emax = std::fmax(cfg.e_max_mev, cfg.mono_energy_mev);
    c->tabs = mcphys::build_tables(0.95 * std::fmin(cfg.photon_cutoff_mev, cfg.wcb_mev), 1.02 * emax,
                                   0.99 * cfg.electron_cutoff_mev, 1.02 * emax, cfg.wcc_mev, cfg.wcb_mev);
    std::vector<float> etab(c->tabs.electron);
    etab.insert(etab.end(), c->tabs.wentzel.begin(), c->tabs.wentzel.end());   // electron kernels stage both
    if (cudaMalloc(&c->d_ptab, sizeof(float) * c->tabs.photon.size()) != cudaSuccess ||
        cudaMalloc(&c->d_etab, sizeof(float) * etab.size()) != cudaSuccess)
        return bail(MC_ERR_OOM);
    cudaMemcpy(c->d_ptab, c->tabs.photon.data(), sizeof(float) * c->tabs.photon.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_etab, etab.data(), sizeof(float) * etab.size(), cudaMemcpyHostToDevice);

    c->cap = cfg.bank_capacity;
    const size_t per = static_cast<size_t>(c->cap) * 4;
    const size_t total = per * 13 * mc::kNumBanks * 2;
    if (cudaMalloc(&c->bank_mem, total) != cudaSuccess) return bail(MC_ERR_OOM);
    char* base = static_cast<char*>(c->bank_mem);
    for (int t = 0; t < mc::kNumBanks; ++t) {
        for (int k = 0; k < 2; ++k) {
            BankPtr& b = c->bank[t][k];
            float** f[8] = {&b.x, &b.y, &b.z, &b.u, &b.v, &b.w, &b.E, &b.tau};
            for (int i = 0; i < 8; ++i) { *f[i] = reinterpret_cast<float*>(base); base += per; }
            uint32_t** q[5] = {&b.hist, &b.ord, &b.draws, &b.cell, &b.flags};
            for (int i = 0; i < 5; ++i) { *q[i] = reinterpret_cast<uint32_t*>(base); base += per; }
        }
    }
    if (cudaMalloc(&c->d_ctl, sizeof(Ctl)) != cudaSuccess || cudaMallocHost(&c->h_ctl, sizeof(Ctl)) != cudaSuccess ||
        cudaMalloc(&c->d_heads, kHeadsBytes) != cudaSuccess ||
        cudaMallocHost(&c->h_fields, sizeof(FieldDev) * mc::kMaxFields) != cudaSuccess ||
        cudaMallocHost(&c->h_first, sizeof(unsigned long long) * (mc::kMaxFields + 1)) != cudaSuccess)
        return bail(MC_ERR_OOM);
    if (cudaEventCreate(&c->ev_run0) != cudaSuccess || cudaEventCreate(&c->ev_run1) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_stage, cudaEventDisableTiming) != cudaSuccess)
        return bail(MC_ERR_CUDA);
    if (cudaMalloc(&c->d_energy, sizeof(unsigned long long) * mc::kNumEnergy) != cudaSuccess ||
        cudaMalloc(&c->d_events, sizeof(unsigned long long) * mc::kNumEvents) != cudaSuccess ||
        cudaMalloc(&c->d_rho_max, sizeof(unsigned int) * 4) != cudaSuccess ||
        cudaMalloc(&c->d_thr, sizeof(float) * 3) != cudaSuccess ||
        cudaMalloc(&c->d_nb, sizeof(double) * cfg.n_batches) != cudaSuccess ||
        cudaMalloc(&c->d_rsum, sizeof(unsigned long long) * cfg.n_batches) != cudaSuccess ||
        cudaMalloc(&c->d_rstat, sizeof(double) * 2) != cudaSuccess ||
        cudaMalloc(&c->d_u, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_maxbits, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_fields, sizeof(FieldDev) * mc::kMaxFields) != cudaSuccess ||
        cudaMalloc(&c->d_first, sizeof(unsigned long long) * (mc::kMaxFields + 1)) != cudaSuccess)
        return bail(MC_ERR_OOM);
    cudaMemset(c->d_energy, 0, sizeof(unsigned long long) * mc::kNumEnergy);
    cudaMemset(c->d_events, 0, sizeof(unsigned long long) * mc::kNumEvents);

    c->block = cfg.block_size;
    if (mc::transport_prepare() != cudaSuccess) return bail(MC_ERR_CUDA);
    for (int t = 0; t < mc::kNumBanks; ++t) {
        int occ = 0;
        c->minb[t] = cfg.regs_variant[t];
        if (mc::transport_occupancy(t, c->minb[t], c->block, &occ) != cudaSuccess || occ < 1) return bail(MC_ERR_CUDA);
        const int per_sm = cfg.ctas_per_sm > 0 ? std::min(cfg.ctas_per_sm, occ) : occ;
        c->grid[t] = c->sm_count * per_sm;
    }
    c->src_grid = c->sm_count * 8;
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(MC_ERR_CUDA);
    *out = c;
    return MC_OK;
}

mc_status mc_destroy(mc_ctx* c) {
    if (!c) return MC_OK;
    cudaSetDevice(c->device);
    finalize_run(c);
    if (c->ev_stage) cudaEventSynchronize(c->ev_stage);
    free_field_buffers(c);
    if (c->h_fields) cudaFreeHost(c->h_fields);
    if (c->h_first) cudaFreeHost(c->h_first);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->ev_run0) cudaEventDestroy(c->ev_run0);
    if (c->ev_run1) cudaEventDestroy(c->ev_run1);
    if (c->ev_stage) cudaEventDestroy(c->ev_stage);
    dfree(c->d_ptab);
    dfree(c->d_etab);
    if (c->bank_mem) cudaFree(c->bank_mem);
    dfree(c->d_ctl);
    dfree(c->d_heads);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    dfree(c->d_hu);
    dfree(c->d_rho);
    dfree(c->d_rho_hom);
    dfree(c->d_hom_tmp);
    dfree(c->d_rho_max);
    dfree(c->d_thr);
    dfree(c->d_mgrid);
    dfree(c->d_energy);
    dfree(c->d_events);
    dfree(c->d_nb);
    dfree(c->d_rsum);
    dfree(c->d_rstat);
    dfree(c->d_u);
    dfree(c->d_maxbits);
    dfree(c->d_fields);
    dfree(c->d_first);
    dfree(c->d_vox);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
    return MC_OK;
}

mc_status mc_init_geometry(mc_ctx* c, const int16_t* hu, int nx, int ny, int nz, const double vox_cm[3],
                           const double origin_cm[3], const mc_epid_desc* epid, int hu_on_device, void* stream) {
    if (!c) return MC_ERR_ARG;
    if (!hu || !vox_cm || !origin_cm || !epid) return fail(c, MC_ERR_ARG, "null pointer");
    if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 1024)
        return fail(c, MC_ERR_ARG, "CT dimensions must be 1..1024 per axis");
    for (int k = 0; k < 3; ++k)
        if (!(vox_cm[k] > 0) || !std::isfinite(origin_cm[k])) return fail(c, MC_ERR_ARG, "bad voxel size or origin");
    const mc_epid_desc& E = *epid;
    if (E.n_layers < 1 || E.n_layers > MC_MAX_LAYERS || E.sensitive_layer < 0 || E.sensitive_layer >= E.n_layers)
        return fail(c, MC_ERR_ARG, "bad EPID layer stack");
    if (E.npx < 1 || E.npy < 1 || E.npx > 8192 || E.npy > 8192 || !(E.pitch_cm > 0))
        return fail(c, MC_ERR_ARG, "bad EPID pixel grid");
    for (int l = 0; l < E.n_layers; ++l)
        if (E.material[l] < 0 || E.material[l] >= MC_NUM_MATERIALS || !(E.thickness_cm[l] > 0) || !(E.density[l] > 0))
            return fail(c, MC_ERR_ARG, "bad EPID layer");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    const mc_status prev = finalize_run(c);          // the CT buffers below may be replaced
    if (prev != MC_OK) return prev;
    clear_fields(c);
    const size_t nvox = static_cast<size_t>(nx) * ny * nz;
    if (nvox > c->nvox_alloc) {
        dfree(c->d_hu);
        dfree(c->d_rho);
        dfree(c->d_rho_hom);
        dfree(c->d_hom_tmp);
        CUDA_TRY(c, cudaMalloc(&c->d_hu, nvox * sizeof(int16_t) + 16));
        CUDA_TRY(c, cudaMalloc(&c->d_rho, nvox * sizeof(float) + 32));
        CUDA_TRY(c, cudaMalloc(&c->d_rho_hom, nvox * sizeof(float) + 32));
        CUDA_TRY(c, cudaMalloc(&c->d_hom_tmp, 2 * nvox * sizeof(int)));
        c->nvox_alloc = nvox;
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_hu, hu, nvox * sizeof(int16_t),
                                hu_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemsetAsync(c->d_rho_max, 0, sizeof(unsigned int) * 4, s));
    CUDA_TRY(c, mc::launch_hu_to_rho(c->d_hu, c->d_rho, nvox, c->d_rho_max, c->d_thr, c->sm_count, s));
    CUDA_TRY(c, mc::launch_homogeneity(c->d_hu, c->d_rho, nx, ny, nz, mc::kHomRadius, mc::kHomSpan, c->d_hom_tmp,
                                       c->d_rho_hom, c->sm_count, s));
    unsigned int bits[4];
    CUDA_TRY(c, cudaMemcpyAsync(bits, c->d_rho_max, sizeof(bits), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->thr, c->d_thr, sizeof(c->thr), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    for (int m = 0; m < 4; ++m) std::memcpy(&c->rho_max[m], &bits[m], sizeof(float));
    // macro-cells: M the smallest power of two >= 4 whose cells are at least
    // kMacroCellCm along every axis and number at most 4096 (measured: cells
    // of ~6 cm beat 3 cm and 13 cm on the 2 mm thorax and the 1 mm
    // anthropomorphic CT)
    int M = 4;
    const double vmin = std::fmin(vox_cm[0], std::fmin(vox_cm[1], vox_cm[2]));   // > 0, checked above
    for (;;) {
        const long cells = static_cast<long>((nx + M - 1) / M) * ((ny + M - 1) / M) * ((nz + M - 1) / M);
        // (a cell as large as the whole CT also ends the search)
        if (cells <= mc::kMaxMacroCells && (M * vmin >= mc::kMacroCellCm || M >= std::max({nx, ny, nz}))) break;
        M *= 2;
    }
    c->mgM = M;
    c->mg[0] = (nx + M - 1) / M; c->mg[1] = (ny + M - 1) / M; c->mg[2] = (nz + M - 1) / M;
    if (!c->d_mgrid) CUDA_TRY(c, cudaMalloc(&c->d_mgrid, sizeof(float2) * mc::kMaxMacroCells));
    CUDA_TRY(c, mc::launch_macro_grid(c->d_rho, nx, ny, nz, M, c->mg[0], c->mg[1], c->mg[2], c->thr[2], c->d_mgrid,
                                      c->sm_count, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (c->cfg.patient_dose && c->vox_n != nvox) {
        dfree(c->d_vox);
        c->vox_n = 0;
        CUDA_TRY(c, cudaMalloc(&c->d_vox, nvox * sizeof(unsigned long long)));
        c->vox_n = nvox;
    }
    if (c->d_vox) CUDA_TRY(c, cudaMemset(c->d_vox, 0, c->vox_n * sizeof(unsigned long long)));
    c->nx = nx; c->ny = ny; c->nz = nz;
    for (int k = 0; k < 3; ++k) { c->vox[k] = vox_cm[k]; c->origin[k] = origin_cm[k]; }
    c->epid = E;
    // layer planes with the sensitive layer's centre at 0; each field puts
    // that centre at its SID
    double z = 0.5 * E.thickness_cm[E.sensitive_layer];
    for (int l = E.sensitive_layer - 1; l >= 0; --l) z += E.thickness_cm[l];
    c->zp[0] = z;
    for (int l = 0; l < E.n_layers; ++l) c->zp[l + 1] = c->zp[l] - E.thickness_cm[l];
    c->has_geom = true;
    return MC_OK;
}

mc_status mc_set_field(mc_ctx* c, const mc_field_desc* f, const mc_lut_desc* lut, void* stream) {
    if (!c) return MC_ERR_ARG;
    if (!f) return fail(c, MC_ERR_ARG, "null field");
    return set_fields_impl(c, f, 1, lut, as_stream(stream));
}

mc_status mc_set_fields(mc_ctx* c, const mc_field_desc* f, int n, const mc_lut_desc* lut, void* stream) {
    if (!c) return MC_ERR_ARG;
    return set_fields_impl(c, f, n, lut, as_stream(stream));
}

mc_status mc_run(mc_ctx* c, uint64_t n, uint64_t seed, void* stream, mc_run_stats* stats) {
    if (!c) return MC_ERR_ARG;
    if (!c->has_field) return fail(c, MC_ERR_STATE, "mc_set_field must come first");
    const std::vector<uint64_t> per(c->fields.size(), n);
    return run_impl(c, per.data(), seed, as_stream(stream), stats);
}

mc_status mc_run_batch(mc_ctx* c, const uint64_t* n, uint64_t seed, void* stream, mc_run_stats* stats) {
    if (!c) return MC_ERR_ARG;
    if (!n) return fail(c, MC_ERR_ARG, "null history counts");
    return run_impl(c, n, seed, as_stream(stream), stats);
}

mc_status mc_get_stats(mc_ctx* c, mc_run_stats* st) {
    if (!c || !st) return MC_ERR_ARG;
    CUDA_TRY(c, cudaSetDevice(c->device));
    const mc_status outcome = finalize_run(c);
    unsigned long long en[mc::kNumEnergy], ev[mc::kNumEvents];
    CUDA_TRY(c, cudaMemcpy(en, c->d_energy, sizeof(en), cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy(ev, c->d_events, sizeof(ev), cudaMemcpyDeviceToHost));
    std::memset(st, 0, sizeof(*st));
    for (const FieldHost& f : c->fields) st->histories += f.hist_done;
    st->e_src_mev = en[mc::kESrc] / kQuantaPerMeV;
    st->e_ct_mev = en[mc::kECT] / kQuantaPerMeV;
    st->e_esc_mev = en[mc::kEEsc] / kQuantaPerMeV;
    st->e_lost_mev = en[mc::kELost] / kQuantaPerMeV;
    for (int l = 0; l < MC_MAX_LAYERS; ++l) st->e_epid_mev[l] = en[mc::kEEpid0 + l] / kQuantaPerMeV;
    for (int k = 0; k < MC_NUM_COUNTERS; ++k) st->counters[k] = ev[k];
    st->waves = c->last_waves;
    st->error_flags = c->last_error;
    st->gpu_ms = c->last_ms;
    for (int t = 0; t < 4; ++t) {
        st->kernel_ms[t] = c->last_kernel_ms[t];
        st->kernel_launches[t] = c->last_kernel_launches[t];
    }
    st->launches = c->last_launches;
    return outcome;
}

mc_status mc_get_field_dose(mc_ctx* c, int field, double* dose, double* sigma, double* u_out, int on_device,
                            void* stream) {
    if (!c) return MC_ERR_ARG;
    mc_status st = check_field(c, field);
    if (st != MC_OK) return st;
    if (!dose) return fail(c, MC_ERR_ARG, "null dose");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    double* dd = on_device ? dose : c->d_dose;
    double* ds = on_device ? (sigma ? sigma : c->d_sigma) : c->d_sigma;
    st = compute_dose(c, field, dd, ds, u_out ? c->d_u : nullptr, s);
    if (st != MC_OK) return st;
    const size_t bytes = sizeof(double) * npix(c);
    if (!on_device) {
        CUDA_TRY(c, cudaMemcpyAsync(dose, c->d_dose, bytes, cudaMemcpyDeviceToHost, s));
        if (sigma) CUDA_TRY(c, cudaMemcpyAsync(sigma, c->d_sigma, bytes, cudaMemcpyDeviceToHost, s));
    }
    if (u_out) CUDA_TRY(c, cudaMemcpyAsync(u_out, c->d_u, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!on_device || u_out) CUDA_TRY(c, cudaStreamSynchronize(s));
    return MC_OK;
}

mc_status mc_get_dose(mc_ctx* c, double* dose, double* sigma, double* u_out, int on_device, void* stream) {
    return mc_get_field_dose(c, 0, dose, sigma, u_out, on_device, stream);
}

mc_status mc_get_field_fluence(mc_ctx* c, int field, double* F, int on_device, void* stream) {
    if (!c) return MC_ERR_ARG;
    mc_status st = check_field(c, field);
    if (st != MC_OK) return st;
    if (!F) return fail(c, MC_ERR_ARG, "null fluence");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    const FieldHost& h = c->fields[field];
    const mc_epid_desc& E = c->epid;
    double* out = on_device ? F : c->d_flu;
    CUDA_TRY(c, mc::launch_fluence(c->d_rect + h.rect_off, c->d_cdf + h.rect_off, h.n_rect, E.npx, E.npy, E.pitch_cm,
                                   h.sid / h.sad, out, s));
    if (!on_device) {
        CUDA_TRY(c, cudaMemcpyAsync(F, c->d_flu, sizeof(double) * npix(c), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    return MC_OK;
}

mc_status mc_get_region_dose(mc_ctx* c, int field, int ix0, int ix1, int iy0, int iy1, double* mean,
                             double* sigma, void* stream) {
    if (!c) return MC_ERR_ARG;
    mc_status st = check_field(c, field);
    if (st != MC_OK) return st;
    if (!mean) return fail(c, MC_ERR_ARG, "null mean");
    if (ix0 < 0 || iy0 < 0 || ix1 <= ix0 || iy1 <= iy0 || ix1 > c->epid.npx || iy1 > c->epid.npy)
        return fail(c, MC_ERR_ARG, "region must be a non-empty pixel rectangle inside the image");
    const int B = c->cfg.n_batches;
    const uint64_t N = c->fields[field].hist_done;
    if (N == 0) return fail(c, MC_ERR_STATE, "no histories run");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    CUDA_TRY(c, mc::launch_batch_counts(c->d_nb, B, N, s));
    const mc_epid_desc& E = c->epid;
    const int l = E.sensitive_layer;
    const double mass_kg = E.density[l] * E.pitch_cm * E.pitch_cm * E.thickness_cm[l] * 1e-3;
    const unsigned long long* tally = c->d_tally + static_cast<size_t>(field) * B * npix(c);
    CUDA_TRY(c, mc::launch_region_stats(tally, E.npx, E.npy, B, c->d_nb, static_cast<double>(N),
                                        kJoulePerMeV / mass_kg, ix0, ix1, iy0, iy1, c->d_rsum, c->d_rstat, s));
    double h[2];
    CUDA_TRY(c, cudaMemcpyAsync(h, c->d_rstat, sizeof(h), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    *mean = h[0];
    if (sigma) *sigma = h[1];
    return MC_OK;
}

mc_status mc_get_field_image(mc_ctx* c, int field, float* signal, int on_device, void* stream) {
    if (!c) return MC_ERR_ARG;
    mc_status st = check_field(c, field);
    if (st != MC_OK) return st;
    if (!c->has_lut) return fail(c, MC_ERR_STATE, "no k-table");
    if (!signal) return fail(c, MC_ERR_ARG, "null signal");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    st = compute_dose(c, field, c->d_dose, c->d_sigma, nullptr, s);
    if (st != MC_OK) return st;
    float* out = on_device ? signal : c->d_signal;
    CUDA_TRY(c, mc::launch_lut(c->d_dose, c->d_tmap + static_cast<size_t>(field) * npix(c), npix(c), c->d_lut_t,
                               c->d_lut_ks + static_cast<size_t>(field) * c->lut_nt, c->lut_nt, c->k_scale, out, s));
    if (!on_device) {
        CUDA_TRY(c, cudaMemcpyAsync(signal, c->d_signal, sizeof(float) * npix(c), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    return MC_OK;
}

mc_status mc_get_epid_image(mc_ctx* c, float* signal, int on_device, void* stream) {
    return mc_get_field_image(c, 0, signal, on_device, stream);
}

mc_status mc_get_field_tmap(mc_ctx* c, int field, double* t, int on_device, void* stream) {
    if (!c) return MC_ERR_ARG;
    mc_status st = check_field(c, field);
    if (st != MC_OK) return st;
    if (!t) return fail(c, MC_ERR_ARG, "null output");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    CUDA_TRY(c, cudaMemcpyAsync(t, c->d_tmap + static_cast<size_t>(field) * npix(c), sizeof(double) * npix(c),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(s));
    return MC_OK;
}

mc_status mc_get_tmap(mc_ctx* c, double* t, int on_device, void* stream) {
    return mc_get_field_tmap(c, 0, t, on_device, stream);
}

mc_status mc_get_tally(mc_ctx* c, uint64_t* tally, int on_device, void* stream) {
    if (!c) return MC_ERR_ARG;
    if (!c->has_field) return fail(c, MC_ERR_STATE, "no field");
    if (!tally) return fail(c, MC_ERR_ARG, "null output");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    CUDA_TRY(c, cudaMemcpyAsync(tally, c->d_tally, sizeof(uint64_t) * c->tally_n,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(s));
    return MC_OK;
}

mc_status mc_get_plan_image(mc_ctx* c, const double* weights, double* dose, double* signal, int on_device,
                            void* stream) {
    if (!c) return MC_ERR_ARG;
    if (!c->has_field) return fail(c, MC_ERR_STATE, "no field");
    if (signal && !c->has_lut) return fail(c, MC_ERR_STATE, "no k-table");
    const int F = nfields(c), np = npix(c);
    for (int f = 0; f < F; ++f)
        if (c->fields[f].hist_done == 0) return fail(c, MC_ERR_STATE, "a field has no histories");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    double *acc_d = nullptr, *acc_s = nullptr;
    CUDA_TRY(c, cudaMalloc(&acc_d, sizeof(double) * np * 2));
    acc_s = acc_d + np;
    cudaError_t e = cudaMemsetAsync(acc_d, 0, sizeof(double) * np * 2, s);
    for (int f = 0; f < F && e == cudaSuccess; ++f) {
        const mc_status st = compute_dose(c, f, c->d_dose, c->d_sigma, nullptr, s);
        if (st != MC_OK) {
            cudaFree(acc_d);
            return st;
        }
        const double w = weights ? weights[f] : 1.0 / F;
        e = mc::launch_plan_accum(c->d_dose, c->d_tmap + static_cast<size_t>(f) * np, np, c->d_lut_t,
                                  c->has_lut ? c->d_lut_ks + static_cast<size_t>(f) * c->lut_nt : nullptr, c->lut_nt,
                                  c->k_scale, w, acc_d, c->has_lut ? acc_s : nullptr, s);
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (e == cudaSuccess && dose) e = cudaMemcpyAsync(dose, acc_d, sizeof(double) * np, kind, s);
    if (e == cudaSuccess && signal) e = cudaMemcpyAsync(signal, acc_s, sizeof(double) * np, kind, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(acc_d);
    if (e != cudaSuccess) return fail(c, MC_ERR_CUDA, std::string("plan image: ") + cudaGetErrorString(e));
    return MC_OK;
}

mc_status mc_get_patient_dose(mc_ctx* c, double* dose, int on_device, void* stream) {
    if (!c) return MC_ERR_ARG;
    if (!dose) return fail(c, MC_ERR_ARG, "null output");
    if (!c->cfg.patient_dose || !c->d_vox || !c->has_geom) return fail(c, MC_ERR_STATE, "patient dose is off");
    uint64_t N = 0;
    for (const FieldHost& f : c->fields) N += f.hist_done;
    if (N == 0) return fail(c, MC_ERR_STATE, "no histories run");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    const double vol = c->vox[0] * c->vox[1] * c->vox[2];
    // Gy per history = E[MeV] * J/MeV / (rho[g/cm^3] V[cm^3] 1e-3 kg/g) / N
    const double conv = kJoulePerMeV / (kQuantaPerMeV * vol * 1e-3 * static_cast<double>(N));
    double* out = dose;
    double* tmp = nullptr;
    if (!on_device) {
        CUDA_TRY(c, cudaMalloc(&tmp, sizeof(double) * c->vox_n));
        out = tmp;
    }
    cudaError_t e = mc::launch_vox_dose(c->d_vox, c->d_rho, c->vox_n, conv, out, s);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(dose, tmp, sizeof(double) * c->vox_n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(c, MC_ERR_CUDA, std::string("patient dose: ") + cudaGetErrorString(e));
    return MC_OK;
}

mc_status mc_get_field_size(mc_ctx* c, int field, double* sz, double* a, double* b) {
    if (!c) return MC_ERR_ARG;
    const mc_status st = check_field(c, field);
    if (st != MC_OK) return st;
    if (sz) *sz = c->fields[field].s_eq;
    if (a) *a = c->fields[field].bbox_a;
    if (b) *b = c->fields[field].bbox_b;
    return MC_OK;
}

mc_status mc_field_size(mc_ctx* c, double* sz, double* a, double* b) { return mc_get_field_size(c, 0, sz, a, b); }

mc_status mc_reset_tally(mc_ctx* c, void* stream) {
    if (!c) return MC_ERR_ARG;
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    const mc_status st = clear_tally(c, s);
    if (st != MC_OK) return st;
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return MC_OK;
}

mc_status mc_state_size(mc_ctx* c, size_t* bytes) {
    if (!c || !bytes) return MC_ERR_ARG;
    if (!c->has_field) return fail(c, MC_ERR_STATE, "no field");
    *bytes = state_words(c) * sizeof(uint64_t);
    return MC_OK;
}

mc_status mc_get_state(mc_ctx* c, void* buf, size_t bytes, void* stream) {
    if (!c || !buf) return MC_ERR_ARG;
    if (!c->has_field) return fail(c, MC_ERR_STATE, "no field");
    if (bytes < state_words(c) * sizeof(uint64_t)) return fail(c, MC_ERR_ARG, "state buffer too small");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    uint64_t* w = static_cast<uint64_t*>(buf);
    const size_t F = c->fields.size();
    w[0] = kStateMagic; w[1] = c->cfg.n_batches; w[2] = c->epid.npx; w[3] = c->epid.npy; w[4] = F;
    w[5] = vox_words(c);
    for (size_t i = 0; i < F; ++i) w[kStateHead + i] = c->fields[i].hist_done;
    uint64_t* q = w + kStateHead + F;
    CUDA_TRY(c, cudaMemcpyAsync(q, c->d_energy, sizeof(uint64_t) * mc::kNumEnergy, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaMemcpyAsync(q + mc::kNumEnergy, c->d_events, sizeof(uint64_t) * mc::kNumEvents,
                                cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaMemcpyAsync(q + mc::kNumEnergy + mc::kNumEvents, c->d_tally, sizeof(uint64_t) * c->tally_n,
                                cudaMemcpyDeviceToHost, s));
    if (vox_words(c))
        CUDA_TRY(c, cudaMemcpyAsync(q + mc::kNumEnergy + mc::kNumEvents + c->tally_n, c->d_vox,
                                    sizeof(uint64_t) * c->vox_n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return MC_OK;
}

mc_status mc_set_state(mc_ctx* c, const void* buf, size_t bytes, void* stream) {
    if (!c || !buf) return MC_ERR_ARG;
    if (!c->has_field) return fail(c, MC_ERR_STATE, "no field");
    if (bytes < state_words(c) * sizeof(uint64_t)) return fail(c, MC_ERR_ARG, "state buffer too small");
    const uint64_t* w = static_cast<const uint64_t*>(buf);
    const size_t F = c->fields.size();
    if (w[0] != kStateMagic || w[1] != static_cast<uint64_t>(c->cfg.n_batches) ||
        w[2] != static_cast<uint64_t>(c->epid.npx) || w[3] != static_cast<uint64_t>(c->epid.npy) || w[4] != F ||
        w[5] != vox_words(c))
        return fail(c, MC_ERR_ARG, "state does not match this context");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = as_stream(stream);
    { const mc_status o = order_after_run(c, s); if (o != MC_OK) return o; }
    const uint64_t* q = w + kStateHead + F;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_energy, q, sizeof(uint64_t) * mc::kNumEnergy, cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_events, q + mc::kNumEnergy, sizeof(uint64_t) * mc::kNumEvents,
                                cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_tally, q + mc::kNumEnergy + mc::kNumEvents, sizeof(uint64_t) * c->tally_n,
                                cudaMemcpyHostToDevice, s));
    if (vox_words(c))
        CUDA_TRY(c, cudaMemcpyAsync(c->d_vox, q + mc::kNumEnergy + mc::kNumEvents + c->tally_n,
                                    sizeof(uint64_t) * c->vox_n, cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    for (size_t i = 0; i < F; ++i) c->fields[i].hist_done = w[kStateHead + i];
    return MC_OK;
}

mc_status mc_set_history_base(mc_ctx* c, uint64_t next_history) {
    if (!c) return MC_ERR_ARG;
    for (FieldHost& f : c->fields) f.hist_done = next_history;
    return MC_OK;
}

mc_status mc_cancel(mc_ctx* c) {
    if (!c) return MC_ERR_ARG;
    c->cancel.store(1);
    return MC_OK;
}

mc_status mc_gamma(const double* ref, const double* ev, int nx, int ny, double pixel_mm, double dd_frac,
                   double dta_mm, double threshold, double step_mm, double radius_mm, double* gamma,
                   double* pass_rate, void* stream) {
    if (!ref || !ev || !pass_rate || nx < 1 || ny < 1 || static_cast<long long>(nx) * ny > (1ll << 28) ||
        !(pixel_mm > 0) || !(dd_frac > 0) || !(dta_mm > 0) || !(threshold >= 0))
        return MC_ERR_ARG;
    const double h = step_mm > 0 ? step_mm : std::fmin(pixel_mm, dta_mm / 10.0);
    const double rad = radius_mm > 0 ? radius_mm : 3.0 * dta_mm;
    if (rad / h > 4096.0) return MC_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    unsigned long long* scratch = nullptr;
    if (cudaMalloc(&scratch, 3 * sizeof(unsigned long long)) != cudaSuccess) return MC_ERR_OOM;
    unsigned long long counts[3] = {0, 0, 0};
    cudaError_t e = mc::launch_gamma(ref, ev, nx, ny, pixel_mm, dd_frac, dta_mm, threshold, h, rad, gamma, scratch, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, scratch, sizeof(counts), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (e != cudaSuccess) return MC_ERR_CUDA;
    *pass_rate = counts[1] ? static_cast<double>(counts[2]) / static_cast<double>(counts[1]) : 1.0;
    return MC_OK;
}

mc_status mc_resample_image(const double* src, int snx, int sny, double src_pitch, double* dst, int dnx, int dny,
                            double dst_pitch, void* stream) {
    if (!src || !dst || snx < 1 || sny < 1 || dnx < 1 || dny < 1 || !(src_pitch > 0) || !(dst_pitch > 0) ||
        static_cast<long long>(dnx) * dny > (1ll << 28))
        return MC_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    if (mc::launch_resample(src, snx, sny, src_pitch, dst, dnx, dny, dst_pitch, s) != cudaSuccess) return MC_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

mc_status mc_test_philox(const uint32_t* in, uint32_t* out, int n, void* stream) {
    if (!in || !out || n < 0) return MC_ERR_ARG;
    if (n == 0) return MC_OK;
    if (mc::launch_test_philox(in, out, n, as_stream(stream)) != cudaSuccess) return MC_ERR_CUDA;
    return cudaStreamSynchronize(as_stream(stream)) == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

mc_status mc_test_uniforms(uint64_t seed, uint64_t hist, uint32_t ord, int n, float* out, void* stream) {
    if (!out || n < 0) return MC_ERR_ARG;
    if (n == 0) return MC_OK;
    if (mc::launch_test_uniforms(seed, hist, ord, n, out, as_stream(stream)) != cudaSuccess) return MC_ERR_CUDA;
    return cudaStreamSynchronize(as_stream(stream)) == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

}  // extern "C"
