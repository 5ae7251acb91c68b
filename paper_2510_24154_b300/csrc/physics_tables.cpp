// Host-side physics data of the CUDA path (see physics_tables.h).
//
// Model (a stated reading; the paper lists the processes in Sec. 2.1.2):
//   Compton        Klein-Nishina per free electron times the electron density.
//   Photoelectric  per atom a Z^4.5 E^-3.2 (a = 4.56e-33 cm^2, E in MeV) with
//                  the Gd K edge at 50.24 keV (jump ratio 5.3).
//   Pair           per atom C Z(Z+1) (1 - 2mc^2/E)^4, C = 2.57e-27 cm^2.
//   Collision      restricted Bethe stopping power (soft Moller losses below
//                  wcc, no density effect) and hard Moller above wcc.
//   Radiative      dsigma/dk = B Z(Z+1) / k per atom, B = 4.65e-27 cm^2,
//                  hard above wcb, continuous below.
//   Scattering     first transport mean free path from the Rossi scattering
//                  power, Es = 21.2 MeV, with the radiation length
//                  4 alpha re^2 N_A sum (w/A) Z(Z+1) ln(183 Z^-1/3).
#include "physics_tables.h"

#include <cmath>

namespace mcphys {
namespace {

struct Element { int Z; double A; };
struct Component { Element el; double w; };
struct MaterialDef { std::vector<Component> parts; double I_eV; };

const Element H{1, 1.008}, C{6, 12.011}, N{7, 14.007}, O{8, 15.999}, Na{11, 22.990}, Mg{12, 24.305},
    P{15, 30.974}, S{16, 32.06}, Cl{17, 35.45}, Ar{18, 39.948}, K{19, 39.098}, Ca{20, 40.078},
    Si{14, 28.085}, Cu{29, 63.546}, Gd{64, 157.25};

const MaterialDef& definition(int m) {
    static const MaterialDef defs[kNumMaterials] = {
        {{{N, 0.755268}, {O, 0.231781}, {Ar, 0.012827}, {C, 0.000124}}, 85.7},                      // air
        {{{H, 0.103}, {C, 0.105}, {N, 0.031}, {O, 0.749}, {Na, 0.002}, {P, 0.002}, {S, 0.003},
          {Cl, 0.003}, {K, 0.002}}, 75.3},                                                          // lung
        {{{H, 0.111894}, {O, 0.888106}}, 75.0},                                                     // water
        {{{H, 0.034}, {C, 0.155}, {N, 0.042}, {O, 0.435}, {Na, 0.001}, {Mg, 0.002}, {P, 0.103},
          {S, 0.003}, {Ca, 0.225}}, 106.4},                                                         // bone
        {{{Cu, 1.0}}, 322.0},                                                                       // copper
        {{{Gd, 0.830790}, {O, 0.084524}, {S, 0.084686}}, 437.0},                                    // Gd2O2S
        {{{Si, 1.0}}, 173.0},                                                                       // a-Si
    };
    return defs[m];
}

constexpr double kPi = 3.14159265358979323846;
constexpr double kPeCoef = 4.56e-33, kPeZ = 4.5;
constexpr double kPairCoef = 2.57e-27;
constexpr double kBremCoef = 4.65e-27;
constexpr double kRossiEs = 21.2;

}  // namespace

MaterialCoefs material_coefs(int m) {
    const MaterialDef& d = definition(m);
    double zA = 0, pe_gd = 0, pe_rest = 0, zz = 0, x0 = 0;
    for (const Component& c : d.parts) {
        const double Z = c.el.Z, per_mol = c.w / c.el.A;
        zA += per_mol * Z;
        (c.el.Z == 64 ? pe_gd : pe_rest) += per_mol * std::pow(Z, kPeZ);
        zz += per_mol * Z * (Z + 1.0);
        x0 += per_mol * Z * (Z + 1.0) * std::log(183.0 / std::cbrt(Z));
    }
    MaterialCoefs r;
    r.zA = zA;
    r.I_MeV = d.I_eV * 1e-6;
    r.ne_barn = kAvogadro * zA * 1e-24;
    r.pe_above = kAvogadro * kPeCoef * (pe_rest + pe_gd);
    r.pe_below = kAvogadro * kPeCoef * (pe_rest + pe_gd / kGdKJump);
    r.pair = kAvogadro * kPairCoef * zz;
    r.brem = kAvogadro * kBremCoef * zz;
    const double inv_x0 = 4.0 * kFineStructure * kRe * kRe * kAvogadro * x0;
    r.msc = 0.5 * kRossiEs * kRossiEs * inv_x0;
    return r;
}

MaterialCoefs tungsten_coefs() {
    const double Z = 74.0, per_mol = 1.0 / 183.84;
    MaterialCoefs r{};
    r.zA = per_mol * Z;
    r.I_MeV = 727e-6;
    r.ne_barn = kAvogadro * r.zA * 1e-24;
    r.pe_above = kAvogadro * kPeCoef * per_mol * std::pow(Z, kPeZ);
    r.pe_below = r.pe_above / kWKJump;
    r.pair = kAvogadro * kPairCoef * per_mol * Z * (Z + 1.0);
    return r;
}

double klein_nishina_barn(double E) {
    // 2 pi re^2 { (1+k)/k^2 [2(1+k)/(1+2k) - ln(1+2k)/k] + ln(1+2k)/(2k) - (1+3k)/(1+2k)^2 }
    const double k = E / kMec2, q = 1.0 + 2.0 * k, lq = std::log(q);
    const double bracket = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / q - lq / k) + lq / (2.0 * k) -
                           (1.0 + 3.0 * k) / (q * q);
    return 2.0 * kPi * kRe * kRe * bracket * 1e24;
}

double pair_shape(double E) {
    const double thr = 2.0 * kMec2;
    if (E <= thr) return 0.0;
    const double r = 1.0 - thr / E;
    return r * r * r * r;
}

double collision_stopping_restricted(int m, double T, double wcc) {
    const MaterialCoefs mc = material_coefs(m);
    const double tau = T / kMec2, gam = tau + 1.0, beta2 = 1.0 - 1.0 / (gam * gam);
    const double cut = std::fmin(wcc, 0.5 * T) / kMec2;   // soft losses stop at the cut (or T/2)
    const double ir = mc.I_MeV / kMec2;
    const double fminus = -1.0 - beta2 + std::log((tau - cut) * cut) + tau / (tau - cut) +
                          (0.5 * cut * cut + (2.0 * tau + 1.0) * std::log(1.0 - cut / tau)) / (gam * gam);
    const double k = 2.0 * kPi * kRe * kRe * kMec2 * kAvogadro * mc.zA / beta2;
    return k * (std::log(2.0 * (tau + 2.0) / (ir * ir)) + fminus);
}

double moller_hard(int m, double T, double wcc) {
    if (T <= 2.0 * wcc) return 0.0;
    const MaterialCoefs mc = material_coefs(m);
    const double tau = T / kMec2, gam = tau + 1.0, beta2 = 1.0 - 1.0 / (gam * gam);
    const double e = wcc / T, cc = (tau / gam) * (tau / gam), b = (2.0 * tau + 1.0) / (gam * gam);
    const double integral = 1.0 / e - 1.0 / (1.0 - e) + (0.5 - e) * cc - b * std::log((1.0 - e) / e);
    return kAvogadro * mc.zA * 2.0 * kPi * kRe * kRe * kMec2 / (beta2 * T) * integral;
}

// Screened-Rutherford law p(mu) = A(1+A)/(mu+A)^2 on mu = (1-cos)/2 has mean
// A[(1+A) ln(1+1/A) - 1]; A(G) solves mean = (1 - exp(-G))/2, by bisection on
// ln A (the mean increases monotonically with A).
double wentzel_screening(double G) {
    const double target = 0.5 * -std::expm1(-G);
    auto mean = [](double A) {
        if (A > 1e3) {   // series in 1/A: 1/2 - 1/(6A) + 1/(12A^2) - 1/(20A^3)
            const double x = 1.0 / A;
            return 0.5 - x / 6.0 + x * x / 12.0 - x * x * x / 20.0;
        }
        return A * ((1.0 + A) * std::log1p(1.0 / A) - 1.0);
    };
    double lo = -80.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mean(std::exp(mid)) < target) lo = mid; else hi = mid;
    }
    return std::exp(0.5 * (lo + hi));
}

Tables build_tables(double e_lo, double e_hi, double t_lo, double t_hi, double wcc, double wcb) {
    Tables t;
    for (int m = 0; m < kNumMaterials; ++m) t.mat[m] = material_coefs(m);

    const double le0 = std::log(e_lo), le1 = std::log(e_hi);
    t.p_lnE0 = le0;
    t.p_inv_dlnE = (kPhotonNodes - 1) / (le1 - le0);
    t.photon.resize(2 * kPhotonNodes);
    for (int i = 0; i < kPhotonNodes; ++i) {
        const double E = std::exp(le0 + i / t.p_inv_dlnE);
        t.photon[2 * i] = static_cast<float>(klein_nishina_barn(E));
        t.photon[2 * i + 1] = static_cast<float>(pair_shape(E));
    }

    // The restricted stopping power and the hard Moller cross section change
    // form at T = 2 wcc (below it every Moller secondary is soft): one node
    // sits exactly there, so no interval straddles the kink (linear
    // interpolation across it erred by 1e-4 in the stopping power and fully in
    // the Moller cross section just above threshold; now 3e-6 and, in the
    // first interval above threshold, 1 %).  The grid keeps one node of slack
    // for the shift.
    double lt0 = std::log(t_lo);
    const double lt1 = std::log(t_hi);
    t.e_inv_dlnT = (kElectronNodes - 2) / (lt1 - lt0);
    const double lk = std::log(2.0 * wcc);
    if (lk > lt0 && lk < lt1) lt0 = lk - std::ceil((lk - lt0) * t.e_inv_dlnT) / t.e_inv_dlnT;
    t.e_lnT0 = lt0;
    t.electron.resize(static_cast<size_t>(kNumMaterials) * 2 * kElectronNodes);
    for (int m = 0; m < kNumMaterials; ++m) {
        for (int i = 0; i < kElectronNodes; ++i) {
            const double T = std::exp(lt0 + i / t.e_inv_dlnT);
            const double soft = collision_stopping_restricted(m, T, wcc) + t.mat[m].brem * std::fmin(wcb, T);
            float* row = &t.electron[(static_cast<size_t>(m) * kElectronNodes + i) * 2];
            row[0] = static_cast<float>(soft);
            row[1] = static_cast<float>(moller_hard(m, T, wcc));
        }
    }
    // ln G from 1e-16 (steps far below the FP32 resolution of a position) to
    // 13.12, just under the isotropic limit ln(5e5) where <1 - cos> is within
    // 2e-6 of 1
    const double lg0 = std::log(1e-16), lg1 = std::log(13.12);
    t.w_lnG0 = lg0;
    t.w_inv_dlnG = (kWentzelNodes - 1) / (lg1 - lg0);
    t.wentzel.resize(kWentzelNodes);
    for (int i = 0; i < kWentzelNodes; ++i)
        t.wentzel[i] = static_cast<float>(std::log(wentzel_screening(std::exp(lg0 + i / t.w_inv_dlnG))));
    return t;
}

}  // namespace mcphys
