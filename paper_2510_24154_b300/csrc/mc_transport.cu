// Transport kernels of the EPID transit Monte Carlo (paper Sec. 2.1).
//
// Four persistent kernels, one per event type, run in waves:
//   photons in the CT    Woodcock (delta) tracking against the majorant
//                        max_m rho_max,m mu_m(E); real interactions sampled as
//                        Compton (Klein-Nishina), photoelectric or pair (Sec. 2.1.2).
//   electrons in the CT  Class II condensed history: CSDA soft losses, hard
//                        Moller and bremsstrahlung by delta tracking against
//                        the start-of-step value, a random-hinge Wentzel
//                        deflection, steps limited by voxel faces; up to four
//                        steps per warp iteration while steps emit nothing.
//   photons in the EPID  exact optical-depth tracking through the layer stack.
//   electrons in the EPID the same condensed history in the layers; energy in
//                        the sensitive layer goes to the pixel tally.
// A source kernel opens each wave: it samples that wave's primaries (Sec.
// 2.1.1) one per thread, with every lane doing the same work, and writes them
// into the CT-photon bank (or the EPID-photon bank when they miss the CT), so
// the transport kernels never branch into history start-up.
// Each kernel follows, draw for draw, the sampling order of the written model,
// so a history fed the same Philox keys replays on another implementation.
#include "mc_device.cuh"
#include "physics_tables.h"

namespace mc {

namespace {

// Per-block accumulators and lane-private counters.
struct Acc {
    unsigned long long ct, src, esc, lost;
    uint32_t flights, steps;
    uint32_t iters, live;       // warp iterations and live lanes (lane 0 counts)
    // EPID kernels: `ct` holds the lane's pending deposit in layer `lay`,
    // added to the block's layer total when the layer changes and at the end
    // (same-address shared atomics from a whole warp on every step would serialise)
    uint32_t lay;
};

__device__ __forceinline__ void acc_flush(const Params& P, Acc& a, unsigned long long* s_energy,
                                          unsigned long long* s_events, int flights_idx, int steps_idx) {
    // warp reduction of the lane-private values, then one shared atomic per warp
    unsigned long long v[4] = {a.ct, a.src, a.esc, a.lost};
    uint32_t f = a.flights, s = a.steps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += __shfl_down_sync(kFull, v[k], o);
        f += __shfl_down_sync(kFull, f, o);
        s += __shfl_down_sync(kFull, s, o);
    }
    if (lane_id() == 0) {
        if (v[0]) atomicAdd(&s_energy[kECT], v[0]);
        if (v[1]) atomicAdd(&s_energy[kESrc], v[1]);
        if (v[2]) atomicAdd(&s_energy[kEEsc], v[2]);
        if (v[3]) atomicAdd(&s_energy[kELost], v[3]);
        if (f) atomicAdd(&s_events[flights_idx], static_cast<unsigned long long>(f));
        if (s) atomicAdd(&s_events[steps_idx], static_cast<unsigned long long>(s));
    }
}

// Adds n per calling lane to event counter idx: the converged lanes that
// reach this call together are counted by one of them with a single shared
// atomic (same-address atomics from many lanes would serialise).
__device__ __forceinline__ void count_event(unsigned long long* s_events, int idx, unsigned n = 1u) {
    const unsigned m = __activemask();
    if (lane_id() == __ffs(m) - 1) atomicAdd(&s_events[idx], static_cast<unsigned long long>(__popc(m) * n));
}

__device__ __forceinline__ float rest_extra(uint32_t flags) { return (flags & kPositron) ? kTwoMec2 : 0.0f; }

// Energy deposited at beam-frame position (x, y) in EPID layer `layer` by a
// particle of history `hist` of field `f`: into sub-tally (history index within the field mod B).
__device__ __forceinline__ void deposit_epid(const Params& P, Acc& a, unsigned long long* s_energy, int layer,
                                             float x, float y, uint32_t hist, uint32_t flags, float dE) {
    if (!(dE > 0.0f)) return;
    const unsigned long long q = quanta(dE);
    if (static_cast<uint32_t>(layer) != a.lay) {
        if (a.ct) atomicAdd(&s_energy[kEEpid0 + a.lay], a.ct);
        a.lay = static_cast<uint32_t>(layer);
        a.ct = 0ull;
    }
    a.ct += q;
    if (layer != P.sens) return;
    int ix = __float2int_rd((x + P.hwx) / P.pitch);
    int iy = __float2int_rd((y + P.hwy) / P.pitch);
    ix = min(max(ix, 0), P.npx - 1);
    iy = min(max(iy, 0), P.npy - 1);
    const FieldDev& F = P.fields[field_of(flags)];
    const unsigned long long b = (F.batch_base + hist) % static_cast<unsigned long long>(P.nbatch);
    atomicAdd(&P.tally[F.tally_off + (b * P.npy + iy) * P.npx + ix], q);
}

template <bool EPID>
__device__ __forceinline__ void deposit(const Params& P, Acc& a, unsigned long long* s_energy, uint32_t cell,
                                        float x, float y, uint32_t hist, uint32_t flags, float dE) {
    if (EPID) {
        deposit_epid(P, a, s_energy, static_cast<int>(cell), x, y, hist, flags, dE);
    } else if (dE > 0.0f) {
        const unsigned long long q = quanta(dE);
        a.ct += q;
        // patient dose: the same quanta into the particle's voxel, so the voxel
        // tally sums to the CT energy exactly
        if (P.vox)
            atomicAdd(&P.vox[(static_cast<size_t>(cell_z(cell)) * P.ny + cell_y(cell)) * P.nx + cell_x(cell)], q);
    }
}

// Sends a particle that leaves the CT across the vacuum gap: onto the EPID's
// top plane if its line meets the detector face, else out of the world.
// Any point of the line will do: the CT lies wholly above the detector.
__device__ __forceinline__ bool transfer_to_epid(const Params& P, Part& p, Acc& a, unsigned long long* s_events,
                                                 bool is_photon) {
    const FieldDev& F = P.fields[field_of(p.flags)];
    float bx, by, bz, bu, bv, bw;
    to_beam(F, p.x, p.y, p.z, bx, by, bz);
    to_beam_dir(F, p.u, p.v, p.w, bu, bv, bw);
    const float eexit = p.E + rest_extra(p.flags);
    const float t = (F.zface - bz) / bw;
    const float X = bx + t * bu, Y = by + t * bv;
    // the line meets the detector face going down (branch-free: a particle
    // that misses it leaves the world and its state is not used again)
    const bool hit = bw < 0.0f && fabsf(X) < P.hwx && fabsf(Y) < P.hwy;
    a.esc += hit ? 0ull : quanta(eexit);
    // inside the detector z is measured from its face, where single precision
    // resolves the 0.29 mm phosphor to ~1e-8 cm (at Z = -50 cm it would be 4e-6 cm)
    p.x = X; p.y = Y; p.z = 0.0f;
    p.u = bu; p.v = bv; p.w = bw;
    p.cell = 0u;
    if (!hit) return false;
    if (is_photon && p.rng.ord == 0u) {
        count_event(s_events, kCPrimAtEPID);
        if (!(p.flags & kCollided)) count_event(s_events, kCUncollided);
    }
    return true;
}

// A secondary charged particle created by `p` (slot `slot`): queued when
// electrons are transported and above the cutoff, otherwise deposited.
template <bool EPID>
__device__ __forceinline__ void charged(const Params& P, Acc& a, unsigned long long* s_energy,
                                        unsigned long long* s_events, const Part& p, Emit& e, float T, float du,
                                        float dv, float dw, uint32_t slot, bool positron) {
    if (P.coupled && T > P.ecut + kStopMargin) {
        e.dest = EPID ? kElectronEPID : kElectronCT;
        e.E = T; e.u = du; e.v = dv; e.w = dw;
        e.ord = child_ordinal(p.rng.ord, p.rng.d, slot);
        e.flags = kCollided | (positron ? kPositron : 0u);
        if (positron) count_event(s_events, kCPositrons);
        else count_event(s_events, kCElectrons);
    } else {
        deposit<EPID>(P, a, s_energy, p.cell, p.x, p.y, p.hist, p.flags, T);
    }
}

// Annihilation at rest of a stopped positron (or a pair positron born at the
// cutoff): two mc^2 photons, isotropic, back to back; slots 0 and 1 after the
// two direction draws.  Encoded as one emission record of count 2.
template <bool EPID>
__device__ __forceinline__ void annihilate(const Params& P, unsigned long long* s_events, Part& p, Emit& e) {
    const float ct = 2.0f * p.rng.u(P.key) - 1.0f;
    float sp, cp;
    azimuth_sincos(p.rng.u(P.key), sp, cp);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    e.dest = EPID ? kPhotonEPID : kPhotonCT;
    e.E = kMec2;
    e.u = st * cp; e.v = st * sp; e.w = ct;
    e.ord = p.rng.ord;          // both children derive from (ord, d) at write time
    // bit 31 marks a back-to-back pair; bits 2..30 hold the parent's draw count
    e.flags = kCollided | 0x80000000u | ((p.rng.d & 0x1fffffffu) << 2);
    count_event(s_events, kCPhotons2, 2u);
}

// Klein-Nishina composition-rejection; returns eps = E'/E and cos(theta).
__device__ __forceinline__ void sample_kn(const PhiloxKey& K, Rng& r, float E, float& eps, float& ct) {
    const float k = E / kMec2;
    const float e0 = 1.0f / (1.0f + 2.0f * k);
    const float a1 = logf(1.0f + 2.0f * k);
    const float a2 = 0.5f * (1.0f - e0 * e0);
    for (int it = 0; it < 4096; ++it) {
        const float r1 = r.u(K), r2 = r.u(K), r3 = r.u(K);
        // both branches of the composition are evaluated and one is kept
        const float ea = expf(-a1 * r2), eb = sqrtf(e0 * e0 + (1.0f - e0 * e0) * r2);
        const float e = (r1 * (a1 + a2) < a1) ? ea : eb;
        const float t = (1.0f - e) / (k * e);
        const float s2 = t * (2.0f - t);
        const float g = 1.0f - e * s2 / (1.0f + e * e);
        if (r3 < g) { eps = e; ct = 1.0f - t; return; }
    }
    eps = 1.0f; ct = 1.0f;
}

// Moller energy fraction on [wcc/T, 1/2]: 1/eps^2 proposal, rejection on the bracket.
__device__ __forceinline__ float sample_moller(const PhiloxKey& K, Rng& r, float T, float wcc) {
    const float tau = T / kMec2, g = tau + 1.0f;
    const float ec = wcc / T, c = tau / g, bb = (2.0f * tau + 1.0f) / (g * g);
    const float gmax = 2.0f - bb + 0.25f * c * c;
    for (int it = 0; it < 4096; ++it) {
        const float r1 = r.u(K), r2 = r.u(K);
        const float eps = ec / (1.0f - r1 * (1.0f - 2.0f * ec));
        const float x = eps / (1.0f - eps);
        const float gv = 1.0f + x * x + c * c * eps * eps - bb * x;
        if (r2 * gmax < gv) return eps;
    }
    return ec;
}

// Source spectrum E = Emax X, X ~ Beta(3/2, 7/2) as G1/(G1+G2) with
// G1 = Exp + N^2/2 and G2 = 3 Exp + N'^2/2 (one Box-Muller pair), redrawn
// below the photon cutoff.  Six draws per attempt.
__device__ __forceinline__ float sample_spectrum(const PhiloxKey& K, Rng& r, float emax, float pcut) {
    for (int it = 0; it < 4096; ++it) {
        const float ua = r.u(K), ub = r.u(K), uc = r.u(K), ud = r.u(K), u1 = r.u(K), u2 = r.u(K);
        const float L = -logf(u1);
        const float c = cospif(2.0f * u2);
        const float g1 = -logf(ua) + L * c * c;
        const float g2 = -logf(ub * uc * ud) + L * (1.0f - c * c);
        const float E = emax * g1 / (g1 + g2);
        if (E >= pcut) return E;
    }
    return emax * 0.3f;
}

// A real photon interaction of p in material m (per-gram partials mc, mp, mq).
// Returns false when the photon is absorbed.
template <bool EPID>
__device__ __forceinline__ bool photon_interact(const Params& P, Acc& a, unsigned long long* s_energy,
                                                unsigned long long* s_events, Part& p, float mc, float mp,
                                                float mq, Emit& e0, Emit& e1) {
    const float tot = mc + mp + mq;
    const float xi = p.rng.u(P.key);
    p.flags |= kCollided;
    if (xi * tot < mc) {
        count_event(s_events, kCCompton);
        float eps, ct;
        sample_kn(P.key, p.rng, p.E, eps, ct);
        float sp, cp;
        azimuth_sincos(p.rng.u(P.key), sp, cp);
        const float E0 = p.E, E1 = eps * E0;
        const float u0 = p.u, v0 = p.v, w0 = p.w;
        rotate_dir(p.u, p.v, p.w, ct, cp, sp);
        const float T = E0 - E1;
        float eu = E0 * u0 - E1 * p.u, ev = E0 * v0 - E1 * p.v, ew = E0 * w0 - E1 * p.w;
        const float n = sqrtf(eu * eu + ev * ev + ew * ew);
        if (n > 0.0f) { eu /= n; ev /= n; ew /= n; } else { eu = u0; ev = v0; ew = w0; }
        charged<EPID>(P, a, s_energy, s_events, p, e0, T, eu, ev, ew, 0u, false);
        p.E = E1;
        if (p.E < P.pcut) {
            deposit<EPID>(P, a, s_energy, p.cell, p.x, p.y, p.hist, p.flags, p.E);
            return false;
        }
        return true;
    }
    if (xi * tot < mc + mp) {
        count_event(s_events, kCPhoto);
        charged<EPID>(P, a, s_energy, s_events, p, e0, p.E, p.u, p.v, p.w, 0u, false);
        return false;
    }
    count_event(s_events, kCPair);
    const float avail = p.E - kTwoMec2;
    const float xu = p.rng.u(P.key);
    const float Tm = xu * avail, Tp = avail - Tm;
    if (P.coupled) {
        charged<EPID>(P, a, s_energy, s_events, p, e0, Tm, p.u, p.v, p.w, 0u, false);
        if (Tp > P.ecut + kStopMargin) {
            charged<EPID>(P, a, s_energy, s_events, p, e1, Tp, p.u, p.v, p.w, 1u, true);
        } else {
            deposit<EPID>(P, a, s_energy, p.cell, p.x, p.y, p.hist, p.flags, Tp);
            annihilate<EPID>(P, s_events, p, e1);
        }
    } else {
        deposit<EPID>(P, a, s_energy, p.cell, p.x, p.y, p.hist, p.flags, Tm + Tp);
        annihilate<EPID>(P, s_events, p, e0);
    }
    return false;
}

// Distance to leave EPID layer l; which = 0 (layer plane), 1 (x edge), 2 (y edge).
__device__ __forceinline__ float epid_dist(const Params& P, const Part& p, int l, int& which) {
    const float zf = (p.w < 0.0f) ? P.zp[l + 1] : P.zp[l];
    const float dz = (p.w != 0.0f) ? (zf - p.z) / p.w : INFINITY;
    const float dx = (p.u != 0.0f) ? ((p.u > 0.0f ? P.hwx : -P.hwx) - p.x) / p.u : INFINITY;
    const float dy = (p.v != 0.0f) ? ((p.v > 0.0f ? P.hwy : -P.hwy) - p.y) / p.v : INFINITY;
    float d = dz; which = 0;
    if (dx < d) { d = dx; which = 1; }
    if (dy < d) { d = dy; which = 2; }
    return fmaxf(d, 0.0f);
}

// Distance to the faces of CT voxel `cell`; axis = 0, 1, 2.  Branch-free:
// the face ahead on each axis is chosen by the sign of the direction, and an
// axis the direction does not move along is never the nearest.
__device__ __forceinline__ float ct_dist(const Params& P, const Part& p, uint32_t cell, int& axis) {
    const int fx = cell_x(cell) + (p.u > 0.0f ? 1 : 0);
    const int fy = cell_y(cell) + (p.v > 0.0f ? 1 : 0);
    const int fz = cell_z(cell) + (p.w > 0.0f ? 1 : 0);
    const float dx = (p.u != 0.0f) ? (P.ox + fx * P.vx - p.x) / p.u : INFINITY;
    const float dy = (p.v != 0.0f) ? (P.oy + fy * P.vy - p.y) / p.v : INFINITY;
    const float dz = (p.w != 0.0f) ? (P.oz + fz * P.vz - p.z) / p.w : INFINITY;
    float d = dx;
    axis = 0;
    if (dy < d) { d = dy; axis = 1; }
    if (dz < d) { d = dz; axis = 2; }
    return fmaxf(d, 0.0f);
}

// ---------------------------------------------------------------------------
// One Woodcock flight of a CT photon with a piecewise-constant majorant: an
// optical depth tau = -ln(xi) is spent across macro-cells, each with majorant
// max(rho_low,c mu_low(E), rho_bone,c mu_bone(E)) (3D-DDA over the cells); where
// it runs out, the tentative collision in the voxel below (kept inside the
// cell) is real with probability Sigma_voxel / Sigma_c.  Returns false when the
// photon leaves the event type (absorbed, escaped, or moved to the EPID: `move`).
__device__ __forceinline__ bool photon_ct_event(const Params& P, const float2* tab, const float2* grid, Acc& a,
                                                unsigned long long* s_energy, unsigned long long* s_events,
                                                Part& p, Emit& e0, Emit& e1, bool& move) {
    const PhotonXS xs = photon_xs(tab, P, p.E);
    float tot[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float c, q, r;
        photon_mu(P, m, xs, c, q, r);
        tot[m] = c + q + r;
    }
    const float mul = fmaxf(tot[0], fmaxf(tot[1], tot[2])), mub = tot[3];
    p.rng.align();
    float tau = -logf(p.rng.u(P.key));
    ++a.flights;
    const int M = P.mgM;
    const float iu = 1.0f / p.u, iv = 1.0f / p.v, iw = 1.0f / p.w;
    int cx = min(max(__float2int_rd((p.x - P.ox) / (M * P.vx)), 0), P.mgx - 1);
    int cy = min(max(__float2int_rd((p.y - P.oy) / (M * P.vy)), 0), P.mgy - 1);
    int cz = min(max(__float2int_rd((p.z - P.oz) / (M * P.vz)), 0), P.mgz - 1);
    // 3D-DDA in the flight's path length t from its start: tx, ty, tz are the
    // values of t at the current cell's exit plane on each axis (the last
    // cell along an axis may be cut short by the CT edge)
    const float x0 = p.x, y0 = p.y, z0 = p.z;
    const int sx = (p.u > 0.0f) ? 1 : -1, sy = (p.v > 0.0f) ? 1 : -1, sz = (p.w > 0.0f) ? 1 : -1;
    auto exit_t = [&](int c, int s, int n, float o, float v, float org, float dir, float inv) {
        if (dir == 0.0f) return INFINITY;
        const int face = (s > 0) ? min((c + 1) * M, n) : c * M;
        return (o + face * v - org) * inv;
    };
    float tx = exit_t(cx, sx, P.nx, P.ox, P.vx, x0, p.u, iu);
    float ty = exit_t(cy, sy, P.ny, P.oy, P.vy, y0, p.v, iv);
    float tz = exit_t(cz, sz, P.nz, P.oz, P.vz, z0, p.w, iw);
    // path length across one whole cell per axis, and where the line leaves
    // the CT on each axis (no cell's exit lies beyond it)
    const float dx = static_cast<float>(M) * P.vx * fabsf(iu);
    const float dy = static_cast<float>(M) * P.vy * fabsf(iv);
    const float dz = static_cast<float>(M) * P.vz * fabsf(iw);
    const float ex = exit_t(sx > 0 ? P.mgx - 1 : 0, sx, P.nx, P.ox, P.vx, x0, p.u, iu);
    const float ey = exit_t(sy > 0 ? P.mgy - 1 : 0, sy, P.ny, P.oy, P.vy, y0, p.v, iv);
    const float ez = exit_t(sz > 0 ? P.mgz - 1 : 0, sz, P.nz, P.oz, P.vz, z0, p.w, iw);
    float t = 0.0f, Sc = 0.0f;
    const int guard = P.mgx + P.mgy + P.mgz + 3;
    bool inside = false;
    for (int it = 0; it < guard; ++it) {
        const float2 g = grid[(cz * P.mgy + cy) * P.mgx + cx];
        Sc = fmaxf(g.x * mul, g.y * mub);
        float tn = tx;
        int ax = 0;
        if (ty < tn) { tn = ty; ax = 1; }
        if (tz < tn) { tn = tz; ax = 2; }
        const float d = fmaxf(tn - t, 0.0f);
        if (tau < Sc * d) {
            t += tau / Sc;
            inside = true;
            break;
        }
        tau -= Sc * d;
        t = fmaxf(tn, t);
        const bool bx = (ax == 0), by = (ax == 1), bz = (ax == 2);
        cx += bx ? sx : 0;
        cy += by ? sy : 0;
        cz += bz ? sz : 0;
        tx = bx ? fminf(tx + dx, ex) : tx;
        ty = by ? fminf(ty + dy, ey) : ty;
        tz = bz ? fminf(tz + dz, ez) : tz;
        if (static_cast<unsigned>(cx) >= static_cast<unsigned>(P.mgx) ||
            static_cast<unsigned>(cy) >= static_cast<unsigned>(P.mgy) ||
            static_cast<unsigned>(cz) >= static_cast<unsigned>(P.mgz)) break;
    }
    p.x = fmaf(t, p.u, x0);
    p.y = fmaf(t, p.v, y0);
    p.z = fmaf(t, p.w, z0);
    if (!inside) {
        move = transfer_to_epid(P, p, a, s_events, true);
        return false;
    }
    // the voxel under the tentative collision, kept inside its macro-cell
    const int ix = min(max(__float2int_rd((p.x - P.ox) / P.vx), cx * M), min((cx + 1) * M, P.nx) - 1);
    const int iy = min(max(__float2int_rd((p.y - P.oy) / P.vy), cy * M), min((cy + 1) * M, P.ny) - 1);
    const int iz = min(max(__float2int_rd((p.z - P.oz) / P.vz), cz * M), min((cz + 1) * M, P.nz) - 1);
    const float rho = __ldg(&P.rho[(static_cast<size_t>(iz) * P.ny + iy) * P.nx + ix]);
    const int m = material_of(P, rho);
    const float tm = (m == 0) ? tot[0] : (m == 1) ? tot[1] : (m == 2) ? tot[2] : tot[3];
    if (!(p.rng.u(P.key) * Sc < rho * tm)) return true;      // virtual
    count_event(s_events, kCRealCT);
    p.cell = pack_cell(ix, iy, iz);
    float mc, mp, mq;
    photon_mu(P, m, xs, mc, mp, mq);
    return photon_interact<false>(P, a, s_energy, s_events, p, mc, mp, mq, e0, e1);
}

// One optical-depth flight of an EPID photon through the layer stack.
__device__ __forceinline__ bool photon_epid_event(const Params& P, const float2* tab, Acc& a,
                                                  unsigned long long* s_energy, unsigned long long* s_events,
                                                  Part& p, Emit& e0, Emit& e1) {
    const PhotonXS xs = photon_xs(tab, P, p.E);
    p.rng.align();
    float tau = -logf(p.rng.u(P.key));
    ++a.flights;
    for (int guard = 0; guard < 4 * kMaxLayers + 8; ++guard) {
        const int l = static_cast<int>(p.cell);
        float c, q, r;
        photon_mu(P, P.lmat[l], xs, c, q, r);
        const float mu = P.lrho[l] * (c + q + r);
        int which;
        const float d = epid_dist(P, p, l, which);
        if (tau < mu * d) {
            const float s = tau / mu;
            p.x += s * p.u; p.y += s * p.v; p.z += s * p.w;
            return photon_interact<true>(P, a, s_energy, s_events, p, c, q, r, e0, e1);
        }
        tau -= mu * d;
        p.x += d * p.u; p.y += d * p.v; p.z += d * p.w;
        if (which != 0) { a.esc += quanta(p.E); return false; }
        const int nl = l + (p.w < 0.0f ? 1 : -1);
        if (nl < 0 || nl >= P.nl) { a.esc += quanta(p.E); return false; }
        p.cell = static_cast<uint32_t>(nl);
    }
    a.lost += quanta(p.E);
    atomicAdd(&s_events[kCLost], 1ull);
    return false;
}

// Where the second segment of a CT hinge step may run through faces: from
// the hinge (p's position and direction, voxel `cell`, homogeneous or not:
// `hom`) for length `len` it ends in voxel `end` (by floor of the end point).
// Returns true if `cell` is homogeneous and `end` lies within kHomRadius
// voxels of it along every axis (and so inside the CT).
constexpr int kMaxLegFaces = 3 * kHomRadius + 1;
__device__ __forceinline__ bool leg_through(const Params& P, const Part& p, uint32_t cell, bool hom, float len,
                                            uint32_t& end) {
    const int ex = __float2int_rd((fmaf(len, p.u, p.x) - P.ox) / P.vx);
    const int ey = __float2int_rd((fmaf(len, p.v, p.y) - P.oy) / P.vy);
    const int ez = __float2int_rd((fmaf(len, p.w, p.z) - P.oz) / P.vz);
    end = pack_cell(min(max(ex, 0), P.nx - 1), min(max(ey, 0), P.ny - 1), min(max(ez, 0), P.nz - 1));
    return hom && abs(ex - cell_x(cell)) <= kHomRadius && abs(ey - cell_y(cell)) <= kHomRadius &&
           abs(ez - cell_z(cell)) <= kHomRadius;
}

// The patient-dose deposits of a CT hinge step whose second segment ran
// through faces: the step's energy e_step split by path length, (s1 + d0) /
// (s1 + len) into the hinge's voxel `cell` (d0: distance to the first face,
// on axis ax0), then each further piece into the voxel it crosses, walked
// face by face from the hinge (p's position and direction), the last piece
// (the remainder) into `end`.
__device__ __forceinline__ void leg_deposit(const Params& P, Acc& a, const Part& p, uint32_t cell, uint32_t end,
                                            float len, float d0, int ax0, float s1, float e_step) {
    int c[3] = {cell_x(cell), cell_y(cell), cell_z(cell)};
    float e = e_step * ((s1 + d0) / (s1 + len));
    deposit<false>(P, a, nullptr, cell, 0.0f, 0.0f, 0u, 0u, e);
    float left = e_step - e, done = d0;
    int ax = ax0;
    Part q = p;
#pragma unroll 1
    for (int k = 1; k < kMaxLegFaces; ++k) {
        const float dir = (ax == 0) ? p.u : (ax == 1) ? p.v : p.w;
        c[ax] += (dir > 0.0f) ? 1 : -1;
        const uint32_t cc = pack_cell(c[0], c[1], c[2]);
        if (cc == end) break;
        q.x = fmaf(done, p.u, p.x); q.y = fmaf(done, p.v, p.y); q.z = fmaf(done, p.w, p.z);
        const float d = ct_dist(P, q, cc, ax);
        if (d >= len - done) break;
        e = e_step * (d / (s1 + len));
        deposit<false>(P, a, nullptr, cc, 0.0f, 0.0f, 0u, 0u, e);
        left -= e;
        done += d;
    }
    deposit<false>(P, a, nullptr, end, 0.0f, 0.0f, 0u, 0u, left);
}

// One condensed-history step of an electron or positron.
//
// Step length: the least of the 5 % energy-loss step (midpoint stopping
// power) and the distance to a hard event (delta tracking against the
// start-of-step cross section); the deflection, with the scattering power at
// the mid-step energy, is drawn once.  Faces: in the CT the hinge is placed on
// that planned step, and a step whose hinge lies beyond the voxel face goes
// straight to the face, deposits at its midpoint, crosses and then deflects
// for the distance travelled; otherwise the step is a random hinge whose
// second segment runs its full length through the faces it meets (its energy
// split among the voxels by path length) if the hinge's voxel is homogeneous
// and the segment ends within kHomRadius voxels of it, else it stops at the
// face.  In the EPID every step that would reach a layer face is
// a face step and second segments stop at faces.  Both kinds run through one
// code path, selecting where they differ, so the warp diverges as little as
// possible.
template <bool EPID>
__device__ __forceinline__ bool electron_event(const Params& P, const float2* tab, Acc& a,
                                               unsigned long long* s_energy, unsigned long long* s_events,
                                               Part& p, Emit& e0, Emit& e1, bool& move, float& rho_c,
                                               bool& hom_c) {
    float rho;
    int m, layer = 0;
    if (EPID) {
        layer = static_cast<int>(p.cell);
        rho = P.lrho[layer];
        m = P.lmat[layer];
    } else {
        rho = rho_c;               // the density of p.cell, loaded (with hom_c) when the electron entered it
        m = material_of(P, rho);
    }
    ++a.steps;
    p.rng.align();
    const MatC& mcst = P.mat[m];
    const float T = p.E;
    // (a) energy-loss step with the midpoint stopping power
    float dEt = P.step_frac * T;
    if (T - dEt < P.tstop) dEt = T - P.ecut;
    const float Tm = T - 0.5f * dEt;
    const float L = rho * electron_tab(tab, P, m, logf(Tm)).x;
    const float sE = dEt / L;
    // (b) distance to the next tentative hard event: the optical depth p.tau,
    // taken when none is pending, is spent against each step's majorant (the
    // start-of-step hard cross section) across steps and faces
    const float lnT = logf(T);
    // hard bremsstrahlung exists only above wcb: A ln(T / wcb) for T > wcb
    const float Sh = rho * (electron_tab(tab, P, m, lnT).y + mcst.brem * fmaxf(lnT - P.ln_wcb, 0.0f));
    const float xt = p.rng.u(P.key);            // drawn every step, used when no depth is pending
    p.tau = (p.tau > 0.0f) ? p.tau : -logf(xt);
    const float sh = p.tau / Sh;
    // (c) cell face
    int ax;
    const float sb = EPID ? epid_dist(P, p, layer, ax) : ct_dist(P, p, p.cell, ax);
    float s = sE;
    int lim = 0;
    if (sh < s) { s = sh; lim = 1; }
    const float xh = p.rng.u(P.key), xmu = p.rng.u(P.key), xph = p.rng.u(P.key);
    if (EPID ? (sb < s) : (xh * s >= sb)) { s = sb; lim = 2; }
    // multiple-scattering deflection for the distance s, at the mid-step energy
    const float Tg = T - 0.5f * dEt * (s / sE);
    const float pc2 = Tg * (Tg + 2.0f * kMec2);
    const float pb2 = pc2 * pc2 / ((Tg + kMec2) * (Tg + kMec2));
    const float G = s * rho * mcst.msc / pb2;
    const float A = wentzel_A(reinterpret_cast<const float*>(tab + kNumMat * kElectronNodes), P, G);
    const float mu = !(G > 0.0f) ? 0.0f : (A < 0.0f) ? xmu : A * xmu / (1.0f - xmu + A);
    float sp, cp;
    azimuth_sincos(xph, sp, cp);
    const bool face = (lim == 2);
    // first segment: the whole step for a face-limited step, else up to the hinge
    const float s1 = face ? s : xh * s;
    const float sd = face ? 0.5f * s : s1;                     // deposit (and stop) point
    const float hx = p.x + sd * p.u, hy = p.y + sd * p.v, hz = p.z + sd * p.w;
    p.x += s1 * p.u; p.y += s1 * p.v; p.z += s1 * p.w;
    const uint32_t hcell = p.cell;
    const float u0 = p.u, v0 = p.v, w0 = p.w;                  // direction before the deflection
    rotate_dir(p.u, p.v, p.w, 1.0f - 2.0f * mu, cp, sp);
    // second segment (hinge steps only): in the CT it runs its full length
    // through the voxels it meets unless it would leave the CT; otherwise it
    // stops at the first face it meets
    float s2 = 0.0f;
    bool crossed = face, through = false;
    int cax = ax, ax2 = 0;
    float sb2 = 0.0f;
    uint32_t ecell = p.cell;
    // direction component across the crossed face: in the EPID face 0 is a layer
    // plane (z) and faces 1, 2 are the lateral edges; in the CT faces 0, 1, 2 are x, y, z
    float cdir = EPID ? w0 : (ax == 0) ? u0 : (ax == 1) ? v0 : w0;
    {
        // evaluated on every lane (a face step's results are not taken): the
        // warp runs this part once either way, without a divergent branch
        sb2 = EPID ? epid_dist(P, p, layer, ax2) : ct_dist(P, p, p.cell, ax2);
        s2 = face ? 0.0f : s - s1;
        const bool cross = !face && s2 >= sb2;
        if (!EPID) through = leg_through(P, p, p.cell, hom_c, s2, ecell) && cross;
        if (cross && !through) {
            s2 = sb2;
            crossed = true;
            cax = ax2;
            cdir = EPID ? p.w : (ax2 == 0) ? p.u : (ax2 == 1) ? p.v : p.w;
        }
        p.x += s2 * p.u; p.y += s2 * p.v; p.z += s2 * p.w;
    }
    const float dE = dEt * ((s1 + s2) / sE);
    const float Tn = T - dE;
    // a hard-event step that ran its full length ends at the tentative event,
    // which consumes the optical depth; any other step spends its path
    const bool at_event = (lim == 1) && !crossed;
    p.tau = at_event ? 0.0f : p.tau - (s1 + s2) * Sh;
    // a step that ends at or below the stopping energy deposits what is left
    // at its hinge (the same deposit as any other step, with Tn added)
    const bool stop = Tn <= P.tstop;
    if (!EPID && through && P.vox && !stop) {
        // patient dose: the step's energy split among the voxels of the second segment
        Part hp = p;
        hp.x = hx; hp.y = hy; hp.z = hz;
        leg_deposit(P, a, hp, hcell, ecell, s2, sb2, ax2, s1, dE);
    } else {
        deposit<EPID>(P, a, s_energy, hcell, hx, hy, p.hist, p.flags, stop ? dE + Tn : dE);
    }
    if (stop) {
        if (p.flags & kPositron) {
            p.x = hx; p.y = hy; p.z = hz; p.cell = hcell;
            annihilate<EPID>(P, s_events, p, e0);
        }
        return false;
    }
    p.E = Tn;
    if (EPID && crossed) {
        const int nl = layer + (cdir < 0.0f ? 1 : -1);          // layers are numbered down the beam (-z)
        if ((cax != 0) || nl < 0 || nl >= P.nl) {
            if (face) { p.u = u0; p.v = v0; p.w = w0; }         // a face-limited step leaves undeflected
            a.esc += quanta(p.E + rest_extra(p.flags));
            return false;
        }
        p.cell = static_cast<uint32_t>(nl);
        return true;
    }
    if (!EPID && (crossed || through)) {
        // the voxel where the step ends: across the face, or where the second
        // segment ran to; every lane that changes voxel loads its density and
        // flag here, for the next step
        uint32_t nc = ecell;
        bool out = false;
        if (crossed) {
            int ix = cell_x(p.cell), iy = cell_y(p.cell), iz = cell_z(p.cell);
            const int stp = (cdir > 0.0f) ? 1 : -1;
            ix += (cax == 0) ? stp : 0;
            iy += (cax == 1) ? stp : 0;
            iz += (cax == 2) ? stp : 0;
            out = ix < 0 || ix >= P.nx || iy < 0 || iy >= P.ny || iz < 0 || iz >= P.nz;
            nc = pack_cell(ix, iy, iz);
        }
        if (out) {
            if (face) { p.u = u0; p.v = v0; p.w = w0; }         // a face-limited step leaves undeflected
            move = transfer_to_epid(P, p, a, s_events, false);
            return false;
        }
        p.cell = nc;
        const size_t v = (static_cast<size_t>(cell_z(nc)) * P.ny + cell_y(nc)) * P.nx + cell_x(nc);
        const float rh = __ldg(&P.rho_hom[v]);
        rho_c = fabsf(rh);
        hom_c = __float_as_int(rh) < 0;
        if (crossed) return true;
    }
    if (!at_event) return true;
    const float lnTn = logf(Tn);
    const float snm = rho * electron_tab(tab, P, m, lnTn).y;
    const float snb = rho * mcst.brem * fmaxf(lnTn - P.ln_wcb, 0.0f);
    if (!(p.rng.u(P.key) * Sh < snm + snb)) return true;      // delta event
    if (p.rng.u(P.key) * (snm + snb) < snm) {
        count_event(s_events, kCMoller);
        const float eps = sample_moller(P.key, p.rng, Tn, P.wcc);
        float sph, cph;
        azimuth_sincos(p.rng.u(P.key), sph, cph);
        const float W = eps * Tn, Tp = Tn - W;
        const float cs = sqrtf(W * (Tn + 2.0f * kMec2) / (Tn * (W + 2.0f * kMec2)));
        const float cpr = sqrtf(Tp * (Tn + 2.0f * kMec2) / (Tn * (Tp + 2.0f * kMec2)));
        float su = p.u, sv = p.v, sw = p.w;
        rotate_dir(su, sv, sw, cs, cph, sph);
        rotate_dir(p.u, p.v, p.w, cpr, -cph, -sph);
        charged<EPID>(P, a, s_energy, s_events, p, e0, W, su, sv, sw, 0u, false);
        p.E = Tp;
    } else {
        count_event(s_events, kCBrem);
        const float k = P.wcb * expf(p.rng.u(P.key) * logf(Tn / P.wcb));
        e0.dest = EPID ? kPhotonEPID : kPhotonCT;
        e0.E = k; e0.u = p.u; e0.v = p.v; e0.w = p.w;
        e0.ord = child_ordinal(p.rng.ord, p.rng.d, 0u);
        e0.flags = kCollided;
        count_event(s_events, kCPhotons2);
        p.E = Tn - k;
    }
    if (p.E <= P.tstop) {
        deposit<EPID>(P, a, s_energy, p.cell, p.x, p.y, p.hist, p.flags, p.E);
        if (p.flags & kPositron) annihilate<EPID>(P, s_events, p, e1);
        return false;
    }
    return true;
}

// Writes an emission record; a count-2 record (annihilation) becomes two
// back-to-back photons with the ordinals of slots 0 and 1.
__device__ __forceinline__ void flush_emission(const Params& P, const Emit& e, const Part& parent, int own_type,
                                               uint32_t own_in, volatile uint32_t* pool_e = nullptr) {
    const bool has = e.dest >= 0;
    if (__ballot_sync(kFull, has) == 0u) return;                // the common case: nothing to write
    const bool pairrec = has && (e.flags & 0x80000000u);
    const unsigned types = __reduce_or_sync(kFull, has ? (1u << e.dest) : 0u);
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int t = 0; t < kNumBanks; ++t) {
        if (!(types & (1u << t))) continue;                     // warp-uniform
        const bool want = (e.dest == t);
        // records per lane: one, or two for a back-to-back pair
        const unsigned one = __ballot_sync(kFull, want), two = __ballot_sync(kFull, want && pairrec);
        const uint32_t total = __popc(one) + __popc(two);
        const uint32_t par = (t == own_type) ? (own_in ^ 1u) : P.ctl->cur[t];
        uint32_t first;
        if (pool_e != nullptr && t == kElectronCT && two == 0u) {
            // CT electrons from the CT-photon kernel: from the warp's slot pool
            first = pool_reserve(want, &P.ctl->count[t][par], pool_e, P.pool_chunk);
        } else {
            uint32_t base = 0;
            if (lane_id() == 0) base = atomicAdd(&P.ctl->count[t][par], total);
            base = __shfl_sync(kFull, base, 0);
            first = base + __popc(one & lt) + __popc(two & lt);
        }
        if (!want) continue;
        const uint32_t n = pairrec ? 2u : 1u;
        const BankPtr b = P.bank[t][par];
        for (uint32_t k = 0; k < n; ++k) {
            const uint32_t slot = first + k;
            const float sg = (k == 0u) ? 1.0f : -1.0f;
            const uint32_t ord = pairrec ? child_ordinal(e.ord, (e.flags >> 2) & 0x1fffffffu, k) : e.ord;
            const uint32_t fl = (pairrec ? kCollided : e.flags) | (parent.flags & kFieldMask);
            if (slot < P.cap) {
                b.x[slot] = parent.x; b.y[slot] = parent.y; b.z[slot] = parent.z;
                b.u[slot] = sg * e.u; b.v[slot] = sg * e.v; b.w[slot] = sg * e.w;
                b.E[slot] = e.E;
                b.tau[slot] = 0.0f;
                b.hist[slot] = parent.hist;
                b.ord[slot] = ord;
                b.draws[slot] = 0u;
                b.cell[slot] = parent.cell;
                b.flags[slot] = fl;
            } else {
                atomicOr(&P.ctl->error, kErrOverflow);
                atomicAdd(&P.energy[kELost], quanta(e.E + rest_extra(fl)));
            }
        }
    }
}

}  // namespace

// Photon transport through a laterally infinite tungsten slab between the
// beam-frame planes Z = zt and zb < zt (source at Z = SAD, beam along -Z):
// flights against mu_W(E), Compton scattering (Klein-Nishina; the photon goes
// on), photoelectric absorption and pair production absorbed in the
// collimator (their electrons and annihilation photons stay in the head).
// (x, y, z) starts on the top plane.  Returns true with the state on the
// bottom plane if the photon leaves there; false if it is absorbed, falls
// below the photon cutoff or leaves through the top.  The oracle's draws.
constexpr float kJawTop = 28.0f;     // jaw slab top, cm from the source
constexpr int kPs1Cap = 100000;      // source photons a history draws at most
constexpr float kMlcTop = 51.0f;     // leaf slab top, cm from the source
__device__ __forceinline__ bool slab_transport(const Params& P, Rng& r, float& x, float& y, float& z, float& u,
                                               float& v, float& w, float& E, float zt, float zb, bool& collided) {
    for (int f = 0; f < P.max_steps; ++f) {
        const PhotonXS xs = photon_xs(P.ptab, P, E);
        const float mc = P.wmat.ne * xs.skn;
        const float mp = (E < P.w_edge ? P.wmat.pe_below : P.wmat.pe_above) * xs.epow;
        const float mq = P.wmat.pair * xs.pair;
        const float tot = mcphys::kWDensity * (mc + mp + mq);
        r.align();
        const float s = -logf(r.u(P.key)) / tot;
        float d = INFINITY;
        if (w < 0.0f) d = (zb - z) / w;
        else if (w > 0.0f) d = (zt - z) / w;
        if (!(s < d)) {
            if (!(w < 0.0f)) return false;
            x = fmaf(d, u, x);
            y = fmaf(d, v, y);
            z = zb;
            return true;
        }
        x = fmaf(s, u, x);
        y = fmaf(s, v, y);
        z = fmaf(s, w, z);
        const float xi = r.u(P.key);
        if (!(xi * (mc + mp + mq) < mc)) return false;          // photoelectric or pair
        float eps, ct, sp, cp;
        sample_kn(P.key, r, E, eps, ct);
        azimuth_sincos(r.u(P.key), sp, cp);
        rotate_dir(u, v, w, ct, cp, sp);
        E *= eps;
        collided = true;
        if (E < P.pcut) return false;
    }
    return false;
}

// Samples the primary of batch history `k` into p (patient frame, at the CT
// entry point) and returns whether it enters the CT; otherwise `move` tells
// whether it reached the EPID face.  The field is the one whose history range
// [first[f], first[f+1]) holds k; the history id within its stream is
// hist_base + k - first[f].
__device__ __forceinline__ bool start_primary(const Params& P, unsigned long long k, Part& p, Acc& a,
                                              unsigned long long* s_events, bool& move) {
    int f = 0;
    {
        int lo = 0, hi = P.n_fields - 1;            // last f with first[f] <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&P.first[mid]) <= k) lo = mid; else hi = mid - 1;
        }
        f = lo;
    }
    const FieldDev& F = P.fields[f];
    const uint32_t idx = static_cast<uint32_t>(k - __ldg(&P.first[f]));
    p.hist = idx;
    p.cell = 0u;
    p.tau = 0.0f;
    p.flags = static_cast<uint32_t>(f) << kFieldShift;
    p.rng.setup(P.key, F.hist_base + idx, 0u, 0u);
    // phase space 2: photons of the source until one leaves the collimator
    // slabs its rectangle's flags name (none without slabs: the first one)
    float bx = 0.0f, by = 0.0f, bz = F.sad, bu = 0.0f, bv = 0.0f, bw = -1.0f;
    bool got = false, scattered = false;
    for (int k = 0; k < kPs1Cap && !got; ++k) {
        // the first rectangle whose cumulative weight exceeds xi (the last if
        // none does): from the cut point of xi, scanned either way, so the
        // result is exactly that of a binary search over the CDF
        const double xi = static_cast<double>(p.rng.u(P.key));
        const double* cdf = P.cdf + F.rect_off;
        int lo = __ldg(&P.guide[F.rect_off + min(static_cast<int>(xi * F.n_rect), F.n_rect - 1)]);
        while (lo > 0 && xi < __ldg(&cdf[lo - 1])) --lo;
        while (lo < F.n_rect - 1 && xi >= __ldg(&cdf[lo])) ++lo;
        const float4 r = __ldg(&P.rect[F.rect_off + lo]);
        const float X = r.x + (r.y - r.x) * p.rng.u(P.key);
        const float Y = r.z + (r.w - r.z) * p.rng.u(P.key);
        p.E = (P.mono_e > 0.0f) ? P.mono_e : sample_spectrum(P.key, p.rng, P.e_max, P.pcut);
        const unsigned flag = (F.leaf_t > 0.0f || F.jaw_t > 0.0f) ? __ldg(&P.rflag[F.rect_off + lo]) : 0u;
        const float nb = sqrtf(X * X + Y * Y + F.sad * F.sad);
        bx = 0.0f; by = 0.0f; bz = F.sad;
        bu = X / nb; bv = Y / nb; bw = -F.sad / nb;
        scattered = false;
        got = true;
        if (flag & 2u) {
            const float zt = F.sad - kJawTop, t = (zt - bz) / bw;
            bx = fmaf(t, bu, bx); by = fmaf(t, bv, by); bz = zt;
            got = slab_transport(P, p.rng, bx, by, bz, bu, bv, bw, p.E, zt, zt - F.jaw_t, scattered);
        }
        if (got && (flag & 1u)) {
            const float zt = F.sad - kMlcTop, t = (zt - bz) / bw;
            bx = fmaf(t, bu, bx); by = fmaf(t, bv, by); bz = zt;
            got = slab_transport(P, p.rng, bx, by, bz, bu, bv, bw, p.E, zt, zt - F.leaf_t, scattered);
        }
    }
    if (!got) { move = false; return false; }       // every source photon stayed in the collimators
    if (scattered) p.flags |= kCollided;
    a.src += quanta(p.E);
    p.x = F.iso[0] + bx * F.ex[0] + by * F.ey[0] + bz * F.ez[0];
    p.y = F.iso[1] + bx * F.ex[1] + by * F.ey[1] + bz * F.ez[1];
    p.z = F.iso[2] + bx * F.ex[2] + by * F.ey[2] + bz * F.ez[2];
    p.u = bu * F.ex[0] + bv * F.ey[0] + bw * F.ez[0];
    p.v = bu * F.ex[1] + bv * F.ey[1] + bw * F.ez[1];
    p.w = bu * F.ex[2] + bv * F.ey[2] + bw * F.ez[2];
    // slab test against the CT box
    const float lo3[3] = {P.ox, P.oy, P.oz};
    const float hi3[3] = {P.ox + P.nx * P.vx, P.oy + P.ny * P.vy, P.oz + P.nz * P.vz};
    const float x3[3] = {p.x, p.y, p.z}, d3[3] = {p.u, p.v, p.w};
    float t0 = -INFINITY, t1 = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d3[k] != 0.0f) {
            float ta = (lo3[k] - x3[k]) / d3[k], tb = (hi3[k] - x3[k]) / d3[k];
            if (ta > tb) { const float t = ta; ta = tb; tb = t; }
            t0 = fmaxf(t0, ta);
            t1 = fminf(t1, tb);
        } else if (x3[k] < lo3[k] || x3[k] > hi3[k]) {
            t0 = INFINITY;
        }
    }
    if (t0 < t1 && t1 > 0.0f) {
        const float t = fmaxf(t0, 0.0f);
        p.x += t * p.u; p.y += t * p.v; p.z += t * p.w;
        return true;
    }
    move = transfer_to_epid(P, p, a, s_events, true);
    return false;
}

// The persistent transport kernel for one event type.
// EPID electrons are few per wave (about one per lane of the grid) and each
// takes tens of dependent steps, so a launch costs the longest chain of steps
// whatever its size.  While more source waves follow and the input holds less
// than an eighth of a bank, the kernel leaves its input for a later wave (the
// producers append to it) and the bank swap keeps it: the chain is paid once
// for several waves.  Every particle still runs (the last source wave and the
// waves that drain the banks never defer), in an order that changes no result
// (per-particle random streams, integer tallies).
__device__ __forceinline__ bool defer_epid_electrons(const Ctl* c, uint32_t cap) {
    return c->allow_flush != 0u && c->count[kElectronEPID][c->cur[kElectronEPID]] < cap / 8u;
}

template <int TYPE, int MINB>
__global__ void __launch_bounds__(256, MINB) k_transport(const Params P) {
    if (TYPE == kElectronEPID && defer_epid_electrons(P.ctl, P.cap)) return;
    constexpr bool kPhoton = (TYPE == kPhotonCT || TYPE == kPhotonEPID);
    constexpr bool kEpid = (TYPE == kPhotonEPID || TYPE == kElectronEPID);
    constexpr int kTabN = kPhoton ? kPhotonNodes : kNumMat * kElectronNodes + kWentzelNodes / 2;
    constexpr int kMoveTo = kPhoton ? kPhotonEPID : kElectronEPID;
    extern __shared__ float2 s_tab[];
    __shared__ unsigned long long s_energy[kNumEnergy];
    __shared__ unsigned long long s_events[kNumEvents];

    const float2* gtab = kPhoton ? P.ptab : P.etab;
    for (int i = threadIdx.x; i < kTabN; i += blockDim.x) s_tab[i] = __ldg(&gtab[i]);
    float2* s_grid = s_tab + kTabN;                 // macro-cell majorants (CT photons only)
    if (TYPE == kPhotonCT) {
        const int ncell = P.mgx * P.mgy * P.mgz;
        for (int i = threadIdx.x; i < ncell; i += blockDim.x) s_grid[i] = __ldg(&P.mgrid[i]);
    }
    for (int i = threadIdx.x; i < kNumEnergy; i += blockDim.x) s_energy[i] = 0ull;
    for (int i = threadIdx.x; i < kNumEvents; i += blockDim.x) s_events[i] = 0ull;
    // CT photons: per-warp slot pools for the two banks every iteration
    // appends to (CT electrons, photons moving to the EPID): next, end of each
    __shared__ uint32_t s_pool[8][4];
    volatile uint32_t* pool_e = nullptr;
    volatile uint32_t* pool_m = nullptr;
    if (TYPE == kPhotonCT) {
        if (threadIdx.x < 8 * 4) (&s_pool[0][0])[threadIdx.x] = 0u;
        pool_e = &s_pool[threadIdx.x >> 5][0];
        pool_m = &s_pool[threadIdx.x >> 5][2];
    }
    __syncthreads();

    const uint32_t in = P.ctl->cur[TYPE];
    const BankPtr bin = P.bank[TYPE][in];
    // a recorded overflow can leave the count above the capacity: never read past the bank
    const uint32_t n_in = min(P.ctl->count[TYPE][in], P.cap);
    const bool may_flush = P.ctl->allow_flush != 0u;
    const uint32_t move_par = kEpid ? 0u : P.ctl->cur[kMoveTo];

    Acc acc = {0ull, 0ull, 0ull, 0ull, 0u, 0u, 0u, 0u, 0u};
    Part p;
    bool alive = false;
    bool in_open = true;
    int steps_here = 0;
    float rho_c = 0.0f;         // electrons in the CT: density of the current voxel
    bool hom_c = false;         // and whether it is homogeneous
    // input segment this warp reads first, and the segments found dry
    int seg = static_cast<int>((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % kHeadShards);
    uint32_t dry = 0u;

    for (;;) {
        bool move = false;
        // refill dead lanes from the input bank (written as a loop of one pass:
        // with this compiler that form gave the CT-electron kernel about 1 %
        // more speed than the equivalent if-block)
#pragma unroll 1
        for (int pass = 0; pass < 1; ++pass) {
            if (!(in_open && __any_sync(kFull, !alive))) break;
            const bool need = !alive;
            // reserve from the current segment; a segment that runs dry sends
            // the warp on to the next one, and the input is closed for the
            // warp once every segment is dry
            const unsigned m = __ballot_sync(kFull, need);
            const uint32_t lo = static_cast<uint32_t>(static_cast<unsigned long long>(n_in) * seg / kHeadShards);
            const uint32_t hi = static_cast<uint32_t>(static_cast<unsigned long long>(n_in) * (seg + 1) / kHeadShards);
            uint32_t base = 0;
            if (lane_id() == __ffs(m) - 1)
                base = atomicAdd(&P.heads[(TYPE * kHeadShards + seg) * kHeadStride], static_cast<uint32_t>(__popc(m)));
            base = lo + __shfl_sync(kFull, base, __ffs(m) - 1);
            const uint32_t slot = base + __popc(m & lanemask_lt());
            const bool got = need && slot < hi;
            if (base + __popc(m) >= hi) {              // this segment is dry (warp-uniform)
                dry |= 1u << seg;
                seg = (seg + 1) % kHeadShards;
                if (dry == (1u << kHeadShards) - 1u) in_open = false;
            }
            if (got) load_part(bin, slot, p, P);
            // a slot reserved by a CT-photon warp but left unused holds no particle
            if (got && !(p.flags & kDead)) {
                alive = true;
                steps_here = 0;
                if (TYPE == kElectronCT) {
                    const size_t v = (static_cast<size_t>(cell_z(p.cell)) * P.ny + cell_y(p.cell)) * P.nx +
                                     cell_x(p.cell);
                    const float rh = __ldg(&P.rho_hom[v]);
                    rho_c = fabsf(rh);
                    hom_c = __float_as_int(rh) < 0;
                }
            }
        }
        const unsigned live = __ballot_sync(kFull, alive);
        if (live == 0u) {
            if (!in_open) break;
            continue;
        }
        if (may_flush && !in_open && __popc(live) <= P.flush_lanes) {
            flush_self(P, alive, TYPE, in ^ 1u, p);
            alive = false;
            break;
        }
        if (lane_id() == 0) { ++acc.iters; acc.live += __popc(live); }
        Emit e0, e1;
        emit_none(e0);
        emit_none(e1);
        if (alive) {
            bool keep = true;
            // electrons in the CT take up to four steps per iteration, going on
            // while a step emits nothing: the iteration's refill, votes and
            // flushes are shared by several steps (measured best at four; the
            // draws are the same as one step per iteration)
            const int reps = (TYPE == kElectronCT) ? 4 : 1;
#pragma unroll 1
            for (int rep = 0; rep < reps; ++rep) {
                if (rep > 0 && !(keep && e0.dest < 0 && e1.dest < 0)) break;
                if (TYPE == kPhotonCT) keep = photon_ct_event(P, s_tab, s_grid, acc, s_energy, s_events, p, e0, e1, move);
                else if (TYPE == kPhotonEPID) keep = photon_epid_event(P, s_tab, acc, s_energy, s_events, p, e0, e1);
                else keep = electron_event<kEpid>(P, s_tab, acc, s_energy, s_events, p, e0, e1, move, rho_c, hom_c);
                if (keep && ++steps_here > P.max_steps) {
                    acc.lost += quanta(p.E + rest_extra(p.flags));
                    atomicAdd(&s_events[kCLost], 1ull);
                    keep = false;
                }
            }
            alive = keep;
        }
        flush_emission(P, e0, p, TYPE, in, pool_e);
        flush_emission(P, e1, p, TYPE, in, pool_e);
        if (!kEpid) flush_self(P, move, kMoveTo, move_par, p, pool_m);
    }
    if (TYPE == kPhotonCT) {
        pool_retire(P, P.bank[kElectronCT][P.ctl->cur[kElectronCT]], pool_e);
        pool_retire(P, P.bank[kPhotonEPID][move_par], pool_m);
    }

    if (kEpid && acc.ct) {
        atomicAdd(&s_energy[kEEpid0 + acc.lay], acc.ct);
        acc.ct = 0ull;
    }
    acc_flush(P, acc, s_energy, s_events, kPhoton ? (kEpid ? kCFlightsEPID : kCFlightsCT) : kCFlightsCT,
              kEpid ? kCEStepsEPID : kCEStepsCT);
    if (!kEpid && lane_id() == 0 && acc.iters) {
        atomicAdd(&s_events[kPhoton ? kCItersPCT : kCItersECT], static_cast<unsigned long long>(acc.iters));
        atomicAdd(&s_events[kPhoton ? kCLivePCT : kCLiveECT], static_cast<unsigned long long>(acc.live));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kNumEnergy; i += blockDim.x)
        if (s_energy[i]) atomicAdd(&P.energy[i], s_energy[i]);
    for (int i = threadIdx.x; i < kNumEvents; i += blockDim.x)
        if (s_events[i]) atomicAdd(&P.events[i], s_events[i]);
}


// The source of one wave: thread-by-thread the primaries of run-local
// histories [src_begin, src_end), each sampled as the transport would have
// sampled it (same draws), written with its draw count into the CT-photon
// bank, or the EPID-photon bank when its line misses the CT.  Grid-stride,
// whole warps per iteration (the bank reservations are warp-aggregated).
__global__ void __launch_bounds__(256) k_source(const Params P) {
    __shared__ unsigned long long s_energy[kNumEnergy];
    __shared__ unsigned long long s_events[kNumEvents];
    for (int i = threadIdx.x; i < kNumEnergy; i += blockDim.x) s_energy[i] = 0ull;
    for (int i = threadIdx.x; i < kNumEvents; i += blockDim.x) s_events[i] = 0ull;
    __syncthreads();
    const unsigned long long begin = P.ctl->src_begin, end = P.ctl->src_end;
    const uint32_t par_ct = P.ctl->cur[kPhotonCT], par_epid = P.ctl->cur[kPhotonEPID];
    Acc acc = {0ull, 0ull, 0ull, 0ull, 0u, 0u, 0u, 0u, 0u};
    const unsigned long long warps = static_cast<unsigned long long>(gridDim.x) * (blockDim.x >> 5);
    const unsigned long long w0 = static_cast<unsigned long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (unsigned long long base = begin + 32ull * w0; base < end; base += 32ull * warps) {
        const unsigned long long idx = base + static_cast<unsigned long long>(lane_id());
        Part p;
        bool enter = false, move = false;
        if (idx < end) enter = start_primary(P, idx, p, acc, s_events, move);
        flush_self(P, enter, kPhotonCT, par_ct, p);
        flush_self(P, move, kPhotonEPID, par_epid, p);
    }
    acc_flush(P, acc, s_energy, s_events, kCFlightsCT, kCEStepsCT);
    __syncthreads();
    for (int i = threadIdx.x; i < kNumEnergy; i += blockDim.x)
        if (s_energy[i]) atomicAdd(&P.energy[i], s_energy[i]);
    for (int i = threadIdx.x; i < kNumEvents; i += blockDim.x)
        if (s_events[i]) atomicAdd(&P.events[i], s_events[i]);
}

// Closes a consumer pass of bank type t: the drained input parity is emptied
// and the carry parity becomes the next input.
__global__ void k_swap(Ctl* c, uint32_t* heads, int t, uint32_t cap) {
    if (t == kElectronEPID && defer_epid_electrons(c, cap)) return;       // input kept for a later wave
    const uint32_t in = c->cur[t];
    c->count[t][in] = 0u;
    for (int k = 0; k < kHeadShards; ++k) heads[(t * kHeadShards + k) * kHeadStride] = 0u;
    c->cur[t] = in ^ 1u;
}

// Opens a wave: the source kernel will start up to `per_wave` more histories,
// no more than the CT-photon bank has room for beside the photons carried
// over, and at most half a bank (their secondaries fill the electron bank).
__global__ void k_wave_begin(Ctl* c, unsigned long long per_wave, uint32_t cap) {
    const uint32_t carried = c->count[kPhotonCT][c->cur[kPhotonCT]];
    unsigned long long room = (carried < cap) ? cap - carried : 0u;
    room = min(room, static_cast<unsigned long long>(cap / 2u));
    unsigned long long lim = c->next_prim + min(per_wave, room);
    if (lim > c->n_total) lim = c->n_total;
    c->src_begin = c->next_prim;
    c->src_end = lim;
    c->next_prim = lim;
    c->prim_limit = lim;
    c->allow_flush = (lim < c->n_total) ? 1u : 0u;
}

// Closes a wave of a graph-driven run: counts it and tells the enclosing
// conditional while-node whether another wave is needed (work left, no error,
// under the wave cap), so the loop ends on the device without a host sync.
__global__ void k_wave_end(Ctl* c, cudaGraphConditionalHandle h, unsigned int max_waves) {
    bool empty = c->next_prim >= c->n_total;
#pragma unroll
    for (int t = 0; t < kNumBanks; ++t) empty = empty && (c->count[t][c->cur[t]] == 0u);
    c->waves += 1u;
    const unsigned int more = (!empty && c->error == 0u && c->waves < max_waves) ? 1u : 0u;
    c->more = more;
    cudaGraphSetConditional(h, more);
}

// ----------------------------------------------------------- launchers ---

size_t transport_smem(int type) {
    const bool photon = (type == kPhotonCT || type == kPhotonEPID);
    size_t n = photon ? kPhotonNodes : kNumMat * kElectronNodes + kWentzelNodes / 2;
    if (type == kPhotonCT) n += kMaxMacroCells;
    return sizeof(float2) * n;
}

// Each event type is built for 2, 3 and 4 resident CTAs of 256 threads per SM
// (register caps 128, 85 and 64); the launch picks one per type.
template <int TYPE>
static const void* fn_for(int minb) {
    switch (minb) {
        case 2: return reinterpret_cast<const void*>(&k_transport<TYPE, 2>);
        case 4: return reinterpret_cast<const void*>(&k_transport<TYPE, 4>);
        default: return reinterpret_cast<const void*>(&k_transport<TYPE, 3>);
    }
}

static const void* transport_fn(int type, int minb) {
    switch (type) {
        case kPhotonCT: return fn_for<kPhotonCT>(minb);
        case kElectronCT: return fn_for<kElectronCT>(minb);
        case kPhotonEPID: return fn_for<kPhotonEPID>(minb);
        default: return fn_for<kElectronEPID>(minb);
    }
}

// Allows each transport kernel its full dynamic shared memory (the CT-photon
// kernel stages 48 KB: photon table and macro-cell majorants).
cudaError_t transport_prepare() {
    for (int t = 0; t < kNumBanks; ++t)
        for (int mb = 2; mb <= 4; ++mb) {
            const cudaError_t e = cudaFuncSetAttribute(transport_fn(t, mb), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       static_cast<int>(transport_smem(t)));
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t transport_occupancy(int type, int minb, int block, int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_fn(type, minb), block,
                                                         transport_smem(type));
}

cudaError_t launch_transport(int type, int minb, const Params& P, int grid, int block, cudaStream_t s) {
    const size_t smem = transport_smem(type);
    void* args[] = {const_cast<Params*>(&P)};
    return cudaLaunchKernel(transport_fn(type, minb), dim3(grid), dim3(block), args, smem, s);
}

cudaError_t launch_swap(Ctl* c, uint32_t* heads, int t, uint32_t cap, cudaStream_t s) {
    k_swap<<<1, 1, 0, s>>>(c, heads, t, cap);
    return cudaGetLastError();
}

cudaError_t launch_wave_end(Ctl* c, cudaGraphConditionalHandle h, unsigned int max_waves, cudaStream_t s) {
    k_wave_end<<<1, 1, 0, s>>>(c, h, max_waves);
    return cudaGetLastError();
}

cudaError_t launch_wave_begin(Ctl* c, unsigned long long per_wave, uint32_t cap, cudaStream_t s) {
    k_wave_begin<<<1, 1, 0, s>>>(c, per_wave, cap);
    return cudaGetLastError();
}

cudaError_t launch_source(const Params& P, int grid, cudaStream_t s) {
    k_source<<<grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace mc
