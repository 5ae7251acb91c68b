// Host-side physics data of the CUDA path: per-material coefficients and the
// energy tables that the transport kernels stage into shared memory.
//
// This is the GPU library's own implementation of the interaction model (the
// paper names the processes of Sec. 2.1.2 but gives no cross sections); it
// shares no code with the CPU oracle.  Everything is evaluated in double and
// rounded to float once, when the tables are filled.
#pragma once

#include <cstdint>
#include <vector>

namespace mcphys {

constexpr int kNumMaterials = 7;
constexpr int kPhotonNodes = 2048;     // ln-uniform photon table nodes
constexpr int kElectronNodes = 512;    // ln-uniform electron table nodes per material
constexpr int kWentzelNodes = 2048;     // ln A of the screening parameter on a ln G grid

constexpr double kMec2 = 0.51099895;   // MeV
constexpr double kRe = 2.8179403262e-13;
constexpr double kAvogadro = 6.02214076e23;
constexpr double kFineStructure = 1.0 / 137.035999084;
constexpr double kGdKEdge = 0.05024;   // MeV
constexpr double kGdKJump = 5.3;

// Per-gram coefficients of one material (float copies go to the kernels).
struct MaterialCoefs {
    double ne_barn;     // N_A * sum(w Z / A) * 1e-24: mu_C/rho = ne_barn * sigma_KN[barn]
    double pe_above;    // mu_PE/rho = pe * E^-3.2 above the Gd K edge
    double pe_below;    // ... and below it
    double pair;        // mu_pair/rho = pair * (1 - 2 mc^2 / E)^4
    double brem;        // hard brems sigma/rho = brem * ln(T / wcb); soft loss = brem * wcb
    double msc;         // 1/lambda1 per rho = msc / (p beta)^2
    double zA;          // sum(w Z / A)
    double I_MeV;       // mean excitation energy
};

MaterialCoefs material_coefs(int m);

// Tungsten of the collimator slabs (photons only): Z 74, A 183.84, K edge at
// 69.525 keV with jump ratio 4.6; pe_above / pe_below straddle that edge.
constexpr double kWKEdge = 0.069525;   // MeV
constexpr double kWKJump = 4.6;
constexpr double kWDensity = 19.3;     // g/cm^3
MaterialCoefs tungsten_coefs();

// Closed forms used to fill the tables.
double klein_nishina_barn(double E);
double pair_shape(double E);
double collision_stopping_restricted(int m, double T, double wcc);
double moller_hard(int m, double T, double wcc);
double wentzel_screening(double G);

struct Tables {
    // photon: (sigma_KN in barn, pair shape) at E_i = exp(lnE0 + i / inv_dlnE)
    std::vector<float> photon;          // 2 * kPhotonNodes
    double p_lnE0 = 0, p_inv_dlnE = 0;
    // electron, per material: (soft stopping power MeV cm^2/g, hard Moller cm^2/g)
    std::vector<float> electron;        // kNumMaterials * 2 * kElectronNodes
    double e_lnT0 = 0, e_inv_dlnT = 0;
    // ln of the Wentzel screening parameter A(G) with <1-cos> = 1 - exp(-G),
    // on ln G from ln(1e-12) to ln(13) (beyond ~13.1 the law is isotropic)
    std::vector<float> wentzel;         // kWentzelNodes
    double w_lnG0 = 0, w_inv_dlnG = 0;
    MaterialCoefs mat[kNumMaterials];
};

// Fill the tables for photon energies [e_lo, e_hi] and electron kinetic
// energies [t_lo, t_hi] with the given hard-event thresholds.
Tables build_tables(double e_lo, double e_hi, double t_lo, double t_hi, double wcc, double wcb);

}  // namespace mcphys
