// Device-side building blocks of the EPID transit Monte Carlo kernels.
//
// Particles live in structure-of-arrays banks, one pair of banks (input and
// carry) per event type: photons in the CT, electrons in the CT, photons in
// the EPID, electrons in the EPID.  Each transport kernel is persistent: a
// warp keeps one particle per lane, advances every live lane by one event per
// iteration and refills dead lanes from its input bank with one atomic per
// warp on one of the bank's 8 segment counters, so the warp stays full while
// work remains.  Secondaries are compacted into the banks of their event type
// with warp ballots and a prefix count.
//
// Random numbers: draw d of the particle with history id h and ordinal o is
// word d mod 4 of Philox4x32-10 (Salmon et al., SC'11) at counter
// (d div 4, o, h_lo, h_hi) under key (seed_lo, seed_hi), mapped to
// ((u >> 9) + 0.5) 2^-23; every electron step and photon flight starts at the
// next multiple of 4.  Secondaries take the ordinal
// fmix32(parent * 0x85EBCA6B + 8 d + slot + 1) (MurmurHash3 finaliser), with d
// the parent's draw count when it creates them, so a history's random
// numbers do not depend on the order in which the GPU processes events.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mc {

constexpr float kMec2 = 0.51099895f;
constexpr float kTwoMec2 = 1.0219979f;
constexpr int kPhotonNodes = 2048;
constexpr int kElectronNodes = 512;
constexpr int kWentzelNodes = 2048;
constexpr int kMaxMacroCells = 4096;
constexpr double kMacroCellCm = 6.0;   // least macro-cell edge (cm) of the Woodcock majorant grid
// Homogeneous CT voxels (electron steps' second segments may cross their faces):
// at least kHomRadius voxels inside the CT, one material and an HU span of at
// most kHomSpan over the (2 kHomRadius + 1)^3 box around them.
constexpr int kHomRadius = 2;
constexpr int kHomSpan = 200;
constexpr int kNumMat = 7;
constexpr int kMaxLayers = 8;
constexpr float kQuantaPerMeV = 2.56e8f;      // tally unit 2^-8 eV
constexpr float kStopMargin = 1e-6f;          // electrons stop at T <= cutoff + this
constexpr unsigned kFull = 0xffffffffu;

enum BankType { kPhotonCT = 0, kElectronCT = 1, kPhotonEPID = 2, kElectronEPID = 3, kNumBanks = 4 };
// A consumer kernel reads its input bank as kHeadShards contiguous segments,
// each with its own read counter on its own 128-byte line (kHeadStride
// words), so the refills of thousands of warps do not all hit one address.
constexpr int kHeadShards = 8;
constexpr int kHeadStride = 32;
enum EnergyCounter { kESrc = 0, kECT = 1, kEEsc = 2, kELost = 3, kEEpid0 = 4, kNumEnergy = 12 };
enum EventCounter {
    kCFlightsCT = 0, kCRealCT, kCCompton, kCPhoto, kCPair, kCEStepsCT, kCEStepsEPID, kCMoller, kCBrem,
    kCPrimAtEPID, kCUncollided, kCLost, kCFlightsEPID, kCElectrons, kCPositrons, kCPhotons2,
    kCItersPCT, kCLivePCT, kCItersECT, kCLiveECT, kNumEvents
};
// kDead marks a bank slot that a warp reserved but left unused (see
// pool_reserve); readers skip it.
enum Flags : uint32_t { kPositron = 1u, kCollided = 2u, kDead = 0x40000000u };
enum ErrorBits : uint32_t { kErrOverflow = 1u, kErrNonFinite = 2u };

struct MatC {
    float ne, pe_above, pe_below, pair, brem, msc;
};

struct BankPtr {
    float *x, *y, *z, *u, *v, *w, *E, *tau;
    uint32_t *hist, *ord, *draws, *cell, *flags;
};

// Run control shared by the kernels of one run (device memory).
struct Ctl {
    unsigned long long next_prim;   // next history (run-local index) to start
    unsigned long long prim_limit;  // histories started so far, through the current wave
    unsigned long long src_begin;   // the source kernel of this wave starts [src_begin, src_end)
    unsigned long long src_end;
    unsigned long long n_total;
    uint32_t count[kNumBanks][2];
    uint32_t cur[kNumBanks];        // input parity per bank type
    uint32_t allow_flush;           // more primaries follow: warps may hand low-occupancy work on
    uint32_t error;
    uint32_t waves;                 // waves completed (graph-driven runs)
    uint32_t more;                  // 1 while work remains (set by the wave-end kernel)
};

// One field of a run: beam frame (axes and isocentre in patient coordinates),
// source distance, beam-frame Z of the detector face, its source rectangles,
// the random-stream id of its first history in this run (hist_base), that
// history's index within the field (batch_base: sub-tally = index mod B) and
// the field's tally offset.
struct FieldDev {
    float ex[3], ey[3], ez[3], iso[3];
    float sad, zface;
    float leaf_t, jaw_t;            // collimator slab thicknesses (cm); 0 = ideal
    int rect_off, n_rect;
    unsigned long long hist_base;
    unsigned long long batch_base;
    unsigned long long tally_off;
};

// Philox4x32-10 round keys of one seed: round r uses (k[2r], k[2r+1]) =
// (seed_lo + r 0x9E3779B9, seed_hi + r 0xBB67AE85).  Kernels get them in their
// parameters, so the rounds read them as constant operands instead of
// keeping the key in registers and bumping it every round.
struct PhiloxKey {
    uint32_t k[20];
};

__host__ __device__ inline PhiloxKey philox_key(unsigned long long seed) {
    PhiloxKey K;
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k[2 * r] = k0;
        K.k[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}

constexpr uint32_t kFieldShift = 8;             // particle flags bits 8..15: field index
constexpr uint32_t kFieldMask = 0xff00u;
constexpr int kMaxFields = 256;

struct Params {
    // CT (patient frame)
    int nx, ny, nz;
    float ox, oy, oz, vx, vy, vz, ivx, ivy, ivz;
    const float* rho;
    // per voxel: the density with the sign bit set where the voxel is homogeneous
    // (electron second segments may cross its faces): one load gives an electron both
    const float* rho_hom;
    float rho_max[4];
    float thr[3];                   // density thresholds lung / water / bone
    int mgM, mgx, mgy, mgz;         // macro-cells: M voxels per side, cells per axis (<= 4096 cells)
    const float2* mgrid;            // per macro-cell (max density of non-bone voxels, of bone voxels)
    // fields: per-field beam frames, sources and tallies; a batch enumerates the
    // histories of all fields one after the other (first[f] .. first[f+1])
    const struct FieldDev* fields;
    int n_fields;
    const unsigned long long* first;    // [n_fields + 1]
    // EPID (beam frame)
    int nl, sens, npx, npy;
    float pitch, ipitch, hwx, hwy;
    float zp[kMaxLayers + 1];       // layer planes relative to the detector face (EPID particles keep z there)
    int lmat[kMaxLayers];
    float lrho[kMaxLayers];
    // source: rectangles and cumulative weights of all fields, concatenated
    const float4* rect;
    const double* cdf;
    // per field, n_rect cut points: guide[rect_off + j] = the first rectangle
    // whose cumulative weight exceeds j / n_rect (where the search starts)
    const uint32_t* guide;
    const unsigned char* rflag;     // per rectangle: bit 0 behind a closed leaf, bit 1 outside the jaws (slabs)
    float e_max, mono_e;
    MatC wmat;                      // tungsten of the collimator slabs (photon coefficients)
    float w_edge;                   // its K edge, MeV
    // physics
    float pcut, ecut, tstop, wcc, wcb, ln_wcb, step_frac;
    int max_steps, coupled, nbatch;
    MatC mat[kNumMat];
    const float2* ptab;
    float p_lnE0, p_idx;
    const float2* etab;             // [kNumMat][kElectronNodes], then kWentzelNodes/2 float2 of ln A
    float e_lnT0, e_idx;
    float w_lnG0, w_idx;
    // run
    unsigned long long seed;
    PhiloxKey key;                  // round keys of `seed`
    unsigned long long* tally;      // [n_fields][B][npy][npx]
    unsigned long long* energy;     // [kNumEnergy]
    unsigned long long* events;     // [kNumEvents]
    unsigned long long* vox;        // patient dose: energy per CT voxel [nz][ny][nx] (2^-8 eV), or null
    Ctl* ctl;
    uint32_t* heads;                // [kNumBanks][kHeadShards][kHeadStride]: read counters of the input segments
    BankPtr bank[kNumBanks][2];
    uint32_t cap;
    int flush_lanes;
    uint32_t pool_chunk;            // CT photons: slots a warp reserves at a time (1: exact reservations)
};

// ------------------------------------------------------------------ RNG ---

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKey& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ K.k[2 * r], lo1, hi0 ^ c.w ^ K.k[2 * r + 1], lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint32_t child_ordinal(uint32_t parent, uint32_t draws, uint32_t slot) {
    return fmix32(parent * 0x85EBCA6Bu + (draws * 8u + slot + 1u));
}

struct Rng {
    uint32_t ord, hlo, hhi, d;
    uint32_t w0, w1, w2, w3;

    __device__ __forceinline__ void setup(const PhiloxKey& K, unsigned long long hist, uint32_t o, uint32_t draws) {
        hlo = static_cast<uint32_t>(hist);
        hhi = static_cast<uint32_t>(hist >> 32);
        ord = o;
        d = draws;
        if (d & 3u) refill(K);
    }
    __device__ __forceinline__ void refill(const PhiloxKey& K) {
        const uint4 r = philox4x32_10(make_uint4(d >> 2, ord, hlo, hhi), K);
        w0 = r.x; w1 = r.y; w2 = r.z; w3 = r.w;
    }
    // Electron steps and photon flights start on a fresh Philox block, so the
    // lanes of a warp refill together.
    __device__ __forceinline__ void align() { d = (d + 3u) & ~3u; }
    __device__ __forceinline__ float u(const PhiloxKey& K) {
        if ((d & 3u) == 0u) refill(K);
        const uint32_t j = d & 3u;
        const uint32_t w = (j == 0u) ? w0 : (j == 1u) ? w1 : (j == 2u) ? w2 : w3;
        ++d;
        return (static_cast<float>(w >> 9) + 0.5f) * 1.1920928955078125e-07f;
    }
};

// ------------------------------------------------------ fixed point -------

__device__ __forceinline__ unsigned long long quanta(float e_mev) {
    return __float2ull_rn(e_mev * kQuantaPerMeV);
}

// ------------------------------------------------------ warp helpers ------

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// Warp-aggregated reservation of slots in a queue counter: every lane of the
// warp must call it; lanes with want=false get no slot.  One atomic per warp.
__device__ __forceinline__ uint32_t warp_reserve(bool want, uint32_t* counter) {
    const unsigned m = __ballot_sync(kFull, want);
    if (m == 0u) return 0u;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane_id() == leader) base = atomicAdd(counter, static_cast<uint32_t>(__popc(m)));
    base = __shfl_sync(kFull, base, leader);
    return base + __popc(m & lanemask_lt());
}

// The same from a warp-private pool of reserved slots (pool[0] next, pool[1]
// end, in shared memory): the counter is touched only when the pool runs
// out, and then for at least `chunk` slots.  Thousands of warps appending to
// one bank every iteration serialise on its counter's address (about 2500
// cycles per reservation measured in the CT-photon kernel); a chunk of 16
// cuts those atomics several-fold.  A lane's records may straddle the old
// pool's tail and the new chunk; slots still pooled when the kernel ends
// are marked kDead by pool_retire.
__device__ __forceinline__ uint32_t pool_reserve(bool want, uint32_t* counter, volatile uint32_t* pool,
                                                 uint32_t chunk) {
    const unsigned m = __ballot_sync(kFull, want);
    if (m == 0u) return 0u;
    const uint32_t total = __popc(m), rank = __popc(m & lanemask_lt());
    const uint32_t next = pool[0], end = pool[1];
    const uint32_t have = end - next;
    uint32_t nb = 0, take = 0;
    if (have < total) {
        take = max(chunk, total - have);
        if (lane_id() == 0) nb = atomicAdd(counter, take);
        nb = __shfl_sync(kFull, nb, 0);
    }
    __syncwarp();
    if (lane_id() == 0) {
        if (have < total) { pool[0] = nb + (total - have); pool[1] = nb + take; }
        else pool[0] = next + total;
    }
    __syncwarp();
    return rank < have ? next + rank : nb + (rank - have);
}

// --------------------------------------------------------- bank I/O -------

struct Part {
    float x, y, z, u, v, w, E;
    float tau;       // charged particles: optical depth left to the next tentative hard event (<= 0: none drawn)
    uint32_t hist, cell, flags;
    Rng rng;
};

__device__ __forceinline__ void load_part(const BankPtr& b, uint32_t i, Part& p, const Params& P) {
    p.x = b.x[i]; p.y = b.y[i]; p.z = b.z[i];
    p.u = b.u[i]; p.v = b.v[i]; p.w = b.w[i];
    p.E = b.E[i];
    p.tau = b.tau[i];
    p.hist = b.hist[i];
    p.cell = b.cell[i];
    p.flags = b.flags[i];
    const int f = static_cast<int>((p.flags & kFieldMask) >> kFieldShift);
    p.rng.setup(P.key, __ldg(&P.fields[f].hist_base) + p.hist, b.ord[i], b.draws[i]);
}

__device__ __forceinline__ void store_part(const BankPtr& b, uint32_t i, const Part& p) {
    b.x[i] = p.x; b.y[i] = p.y; b.z[i] = p.z;
    b.u[i] = p.u; b.v[i] = p.v; b.w[i] = p.w;
    b.E[i] = p.E;
    b.tau[i] = p.tau;
    b.hist[i] = p.hist;
    b.ord[i] = p.rng.ord;
    b.draws[i] = p.rng.d;
    b.cell[i] = p.cell;
    b.flags[i] = p.flags;
}

// A secondary waiting to be written to a bank at the end of an iteration; it
// starts at its parent's position and cell.
struct Emit {
    int dest;        // bank type, -1 = none
    float E, u, v, w;
    uint32_t ord, flags;
};

__device__ __forceinline__ void emit_none(Emit& e) { e.dest = -1; }

// Moves the lane's own particle into bank `t` (input parity of t), from the
// warp's slot pool when one is given.
__device__ __forceinline__ void flush_self(const Params& P, bool want, int t, uint32_t par, const Part& p,
                                           volatile uint32_t* pool = nullptr) {
    if (__ballot_sync(kFull, want) == 0u) return;
    const uint32_t slot = pool ? pool_reserve(want, &P.ctl->count[t][par], pool, P.pool_chunk)
                               : warp_reserve(want, &P.ctl->count[t][par]);
    if (want) {
        if (slot < P.cap) {
            store_part(P.bank[t][par], slot, p);
        } else {
            atomicOr(&P.ctl->error, kErrOverflow);
            atomicAdd(&P.energy[kELost], quanta(p.E + ((p.flags & kPositron) ? kTwoMec2 : 0.0f)));
        }
    }
}

// Marks the slots still in a warp's pool (below the capacity) as unused.
__device__ __forceinline__ void pool_retire(const Params& P, const BankPtr& b, volatile uint32_t* pool) {
    const uint32_t next = pool[0], end = pool[1];
    for (uint32_t s = next + static_cast<uint32_t>(lane_id()); s < end; s += 32u)
        if (s < P.cap) b.flags[s] = kDead;
    __syncwarp();
}

// -------------------------------------------------------- geometry --------

__device__ __forceinline__ void to_beam(const FieldDev& F, float px, float py, float pz, float& bx, float& by,
                                        float& bz) {
    const float dx = px - F.iso[0], dy = py - F.iso[1], dz = pz - F.iso[2];
    bx = dx * F.ex[0] + dy * F.ex[1] + dz * F.ex[2];
    by = dx * F.ey[0] + dy * F.ey[1] + dz * F.ey[2];
    bz = dx * F.ez[0] + dy * F.ez[1] + dz * F.ez[2];
}

__device__ __forceinline__ void to_beam_dir(const FieldDev& F, float u, float v, float w, float& bu, float& bv,
                                            float& bw) {
    bu = u * F.ex[0] + v * F.ex[1] + w * F.ex[2];
    bv = u * F.ey[0] + v * F.ey[1] + w * F.ey[2];
    bw = u * F.ez[0] + v * F.ez[1] + w * F.ez[2];
}

__device__ __forceinline__ int field_of(uint32_t flags) { return static_cast<int>((flags & kFieldMask) >> kFieldShift); }

__device__ __forceinline__ uint32_t pack_cell(int ix, int iy, int iz) {
    return static_cast<uint32_t>(ix) | (static_cast<uint32_t>(iy) << 10) | (static_cast<uint32_t>(iz) << 20);
}
__device__ __forceinline__ int cell_x(uint32_t c) { return c & 1023u; }
__device__ __forceinline__ int cell_y(uint32_t c) { return (c >> 10) & 1023u; }
__device__ __forceinline__ int cell_z(uint32_t c) { return (c >> 20) & 1023u; }

__device__ __forceinline__ int material_of(const Params& P, float rho) {
    return (rho >= P.thr[0]) + (rho >= P.thr[1]) + (rho >= P.thr[2]);
}

// Sine and cosine of the azimuth 2 pi x of a uniform x in (0, 1), from the
// hardware's approximate sine and cosine (absolute error below 2^-21 on
// [-pi, pi]) of the argument shifted into that range: x - 1/2 is exact for
// the generator's uniforms, and sin, cos of 2 pi x - pi are minus those of 2 pi x.
__device__ __forceinline__ void azimuth_sincos(float x, float& s, float& c) {
    float sn, cs;
    __sincosf(6.28318530717958648f * (x - 0.5f), &sn, &cs);
    s = -sn;
    c = -cs;
}

// Unit direction rotated by polar cosine ct and azimuth (cp, sp); the polar
// frame is used within 0.99999 of the z axis.
__device__ __forceinline__ void rotate_dir(float& u, float& v, float& w, float ct, float cp, float sp) {
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    if (fabsf(w) > 0.99999f) {
        const float sg = (w > 0.0f) ? 1.0f : -1.0f;
        u = st * cp; v = st * sp; w = sg * ct;
    } else {
        const float q = 1.0f - w * w;                           // sin^2 of the polar angle of (u, v, w)
        const float iq = rsqrtf(q);
        const float sq = st * iq;
        const float nu = u * ct + sq * (u * w * cp - v * sp);
        const float nv = v * ct + sq * (v * w * cp + u * sp);
        const float nw = w * ct - q * iq * st * cp;
        u = nu; v = nv; w = nw;
    }
    const float inv = rsqrtf(u * u + v * v + w * w);
    u *= inv; v *= inv; w *= inv;
}

// ------------------------------------------------------- physics ----------

// Photon cross-section components at energy E from the shared-memory table.
struct PhotonXS { float skn, pair, epow; bool below_edge; };

__device__ __forceinline__ PhotonXS photon_xs(const float2* tab, const Params& P, float E) {
    const float lnE = logf(E);
    const float x = (lnE - P.p_lnE0) * P.p_idx;
    const int i = min(max(__float2int_rd(x), 0), kPhotonNodes - 2);
    const float f = x - static_cast<float>(i);
    const float2 a = tab[i], b = tab[i + 1];
    PhotonXS r;
    r.skn = fmaf(f, b.x - a.x, a.x);
    r.pair = fmaf(f, b.y - a.y, a.y);
    r.epow = expf(-3.2f * lnE);
    r.below_edge = E < 0.05024f;
    return r;
}

// Per-gram partial coefficients (Compton, photoelectric, pair) of material m.
__device__ __forceinline__ void photon_mu(const Params& P, int m, const PhotonXS& x, float& mc, float& mp,
                                          float& mq) {
    const MatC& c = P.mat[m];
    mc = c.ne * x.skn;
    mp = (x.below_edge ? c.pe_below : c.pe_above) * x.epow;
    mq = c.pair * x.pair;
}

// Electron table lookup: (soft stopping power, hard Moller) per gram.
__device__ __forceinline__ float2 electron_tab(const float2* tab, const Params& P, int m, float lnT) {
    const float x = (lnT - P.e_lnT0) * P.e_idx;
    const int i = min(max(__float2int_rd(x), 0), kElectronNodes - 2);
    const float f = x - static_cast<float>(i);
    const float2 a = tab[m * kElectronNodes + i], b = tab[m * kElectronNodes + i + 1];
    return make_float2(fmaf(f, b.x - a.x, a.x), fmaf(f, b.y - a.y, a.y));
}

// Screening parameter A of the screened-Rutherford (Wentzel) law whose mean
// <1 - cos> equals 1 - exp(-G); -1 means isotropic (1/2 - <(1 - cos)/2> =
// exp(-G)/2 below 1e-6, i.e. G > ln(5e5)).  Linear interpolation of ln A on a
// 2048-node ln G table in shared memory (after the electron tables): relative
// error below 2e-3 everywhere and 3e-5 on average against the root of the
// defining equation, the same fixed work on every lane.
__device__ __forceinline__ float wentzel_A(const float* wtab, const Params& P, float G) {
    const float x = (logf(fminf(G, 13.1223634f)) - P.w_lnG0) * P.w_idx;
    const int i = min(max(__float2int_rd(x), 0), kWentzelNodes - 2);
    const float f = x - static_cast<float>(i);
    const float A = expf(fmaf(f, wtab[i + 1] - wtab[i], wtab[i]));
    return (G > 13.1223634f) ? -1.0f : A;
}

}  // namespace mc
