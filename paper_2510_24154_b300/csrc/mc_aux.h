// Host-callable launchers of the library's kernels (internal header).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace mc {

struct Params;
struct Ctl;

// Ray-sum arguments for the radiological thickness map.
struct TmapArgs {
    int nx, ny, nz;
    float ox, oy, oz, vx, vy, vz;
    const float* rho;
    float src[3], iso[3], ex[3], ey[3], ez[3];
    int npx, npy;
    float pitch, hwx, hwy, zs;
    double t_offset;
};

size_t transport_smem(int type);
cudaError_t transport_prepare();
cudaError_t transport_occupancy(int type, int minb, int block, int* blocks_per_sm);
cudaError_t launch_transport(int type, int minb, const Params& P, int grid, int block, cudaStream_t s);
cudaError_t launch_swap(Ctl* c, uint32_t* heads, int t, uint32_t cap, cudaStream_t s);
cudaError_t launch_wave_begin(Ctl* c, unsigned long long per_wave, uint32_t cap, cudaStream_t s);
cudaError_t launch_source(const Params& P, int grid, cudaStream_t s);
cudaError_t launch_wave_end(Ctl* c, cudaGraphConditionalHandle h, unsigned int max_waves, cudaStream_t s);

cudaError_t launch_hu_to_rho(const int16_t* hu, float* rho, size_t n, unsigned int* rho_max_bits, float* thr,
                             int sm_count, cudaStream_t s);
// Homogeneity flags of the CT for the electron transport, stored as the sign
// bit of a copy of the density (rho_hom[v] = -rho[v] where homogeneous, so one
// 4-byte load gives an electron entering a voxel both): voxel v is homogeneous
// when it lies at least `radius` voxels inside the CT and the (2 radius + 1)^3
// box around it holds one material with HU values (clamped to [-1024, 3071])
// spanning at most `span`.  tmp: two int32 buffers of n voxels each (scratch).
cudaError_t launch_homogeneity(const int16_t* hu, const float* rho, int nx, int ny, int nz, int radius, int span,
                               int* tmp, float* rho_hom, int sm_count, cudaStream_t s);
cudaError_t launch_macro_grid(const float* rho, int nx, int ny, int nz, int M, int mgx, int mgy, int mgz,
                              float thr_bone, float2* grid, int sm_count, cudaStream_t s);
cudaError_t launch_tmap(const TmapArgs& A, double* t, cudaStream_t s);
// nb[b] = the number of history indices 0 .. n-1 with index mod B == b.
cudaError_t launch_batch_counts(double* nb, int B, unsigned long long n, cudaStream_t s);
// Source-position density (cm^-2 at the isocentre plane) at each EPID pixel
// centre projected by 1 / mag = SAD / SID, from a field's source rectangles
// and their normalised cumulative weights; F[npy][npx] is overwritten.
cudaError_t launch_fluence(const float4* rect, const double* cdf, int n_rect, int npx, int npy, double pitch,
                           double mag, double* F, cudaStream_t s);
// Mean dose per history over pixels [ix0, ix1) x [iy0, iy1) and its batch
// standard error into out[0], out[1]; sums is B words of scratch.
cudaError_t launch_region_stats(const unsigned long long* tally, int npx, int npy, int B, const double* nb,
                                double n_hist, double conv, int ix0, int ix1, int iy0, int iy1,
                                unsigned long long* sums, double* out, cudaStream_t s);
cudaError_t launch_dose(const unsigned long long* tally, int npix, int B, const double* nb, double n_hist,
                        double conv, double* dose, double* sigma, unsigned long long* max_bits, double* part_sum,
                        unsigned int* part_cnt, double* u, cudaStream_t s);
cudaError_t launch_lut(const double* dose, const double* t, int npix, const double* tn, const double* ks, int nt,
                       double k_scale, float* signal, cudaStream_t s);
cudaError_t launch_plan_accum(const double* dose, const double* t, int npix, const double* tn, const double* ks,
                              int nt, double k_scale, double w, double* acc_dose, double* acc_signal, cudaStream_t s);
cudaError_t launch_resample(const double* src, int snx, int sny, double sp, double* dst, int dnx, int dny, double dp,
                            cudaStream_t s);
// dose[v] = vox[v] * conv / rho[v] (patient dose)
cudaError_t launch_vox_dose(const unsigned long long* vox, const float* rho, size_t n, double conv, double* dose,
                            cudaStream_t s);
// scratch: 3 device u64 (max bits, evaluated count, passed count)
cudaError_t launch_gamma(const double* ref, const double* ev, int nx, int ny, double pix, double dd_frac, double dta,
                         double thr_frac, double h, double rad, double* gam, unsigned long long* scratch,
                         cudaStream_t s);
cudaError_t launch_test_philox(const uint32_t* in, uint32_t* out, int n, cudaStream_t s);
cudaError_t launch_test_uniforms(unsigned long long seed, unsigned long long hist, uint32_t ord, int n, float* out,
                                 cudaStream_t s);

}  // namespace mc
