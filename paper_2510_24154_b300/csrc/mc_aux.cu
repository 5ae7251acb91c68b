// Streaming kernels around the transport: HU -> density (Sec. 2.1.2),
// radiological thickness ray sums (Sec. 2.2), dose statistics over the batch
// sub-tallies (Sec. 2.3) and the k(t, s) dose-to-signal correction (Sec. 3.1),
// plus two diagnostics.
#include "mc_aux.h"

#include <algorithm>
#include "mc_device.cuh"

namespace mc {

// ---------------------------------------------- HU -> density --------
// HU-to-density curve (Sec. 2.1.2; the curve itself is a stated reading):
// rho = 1 + HU/1000 for HU <= 0, 1 + 0.6 HU/1000 above, floored at air's
// 0.001205, HU clamped to [-1024, 3071].  Material follows from density
// thresholds evaluated with the same single-precision expression, which is
// strictly increasing in HU, so the class boundaries -900 / -200 / 300 HU are
// reproduced exactly.
__device__ __forceinline__ float rho_of_hu(int hu) {
    hu = min(max(hu, -1024), 3071);
    const float h = static_cast<float>(hu);
    const float r = (hu <= 0) ? fmaf(h, 1e-3f, 1.0f) : fmaf(h, 6e-4f, 1.0f);
    return fmaxf(r, 0.001205f);
}

// Per macro-cell (M^3 voxels) maxima of the non-bone and the bone densities:
// the local Woodcock majorants.  Positive floats order like their bit patterns.
__global__ void k_macro_grid(const float* __restrict__ rho, int nx, int ny, int nz, int M, int mgx, int mgy,
                             float thr_bone, unsigned int* __restrict__ grid) {
    const size_t n = static_cast<size_t>(nx) * ny * nz;
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;      // a multiple of 32
    const unsigned lane = threadIdx.x & 31u;
    // whole warps per pass: lanes with the same (cell, class) reduce their
    // maximum first, and one of them updates the grid (32 consecutive voxels
    // share at most a few cells)
    for (size_t base = static_cast<size_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        const size_t i = base + lane;
        unsigned key = 0xffffffffu, bits = 0u;
        if (i < n) {
            const int ix = static_cast<int>(i % nx), iy = static_cast<int>((i / nx) % ny),
                      iz = static_cast<int>(i / (static_cast<size_t>(nx) * ny));
            const float r = rho[i];
            const size_t cc = (static_cast<size_t>(iz / M) * mgy + iy / M) * mgx + ix / M;
            key = static_cast<unsigned>(2 * cc + (r >= thr_bone ? 1 : 0));
            bits = __float_as_uint(r);
        }
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const unsigned mx = __reduce_max_sync(grp, bits);
        if (i < n && lane == static_cast<unsigned>(__ffs(grp) - 1)) atomicMax(&grid[key], mx);
    }
}

__global__ void k_hu_to_rho(const int16_t* __restrict__ hu, float* __restrict__ rho, size_t n,
                            unsigned int* rho_max_bits, float* thr) {
    __shared__ unsigned int s_max[4];
    if (threadIdx.x < 4) s_max[threadIdx.x] = 0u;
    __syncthreads();
    const float t0 = rho_of_hu(-900), t1 = rho_of_hu(-200), t2 = rho_of_hu(300);
    unsigned int lmax[4] = {0u, 0u, 0u, 0u};
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    // eight voxels per 16-byte load
    const size_t n8 = n / 8;
    const int4* hu8 = reinterpret_cast<const int4*>(hu);
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n8; i += stride) {
        const int4 q = __ldg(&hu8[i]);
        const int32_t w[4] = {q.x, q.y, q.z, q.w};
        float r[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            r[2 * k] = rho_of_hu(static_cast<int16_t>(w[k] & 0xffff));
            r[2 * k + 1] = rho_of_hu(static_cast<int16_t>(static_cast<uint32_t>(w[k]) >> 16));
        }
        float4* out = reinterpret_cast<float4*>(rho + 8 * i);
        out[0] = make_float4(r[0], r[1], r[2], r[3]);
        out[1] = make_float4(r[4], r[5], r[6], r[7]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int m = (r[k] >= t0) + (r[k] >= t1) + (r[k] >= t2);
            const unsigned int b = __float_as_uint(r[k]);
            lmax[0] = (m == 0) ? max(lmax[0], b) : lmax[0];
            lmax[1] = (m == 1) ? max(lmax[1], b) : lmax[1];
            lmax[2] = (m == 2) ? max(lmax[2], b) : lmax[2];
            lmax[3] = (m == 3) ? max(lmax[3], b) : lmax[3];
        }
    }
    for (size_t i = 8 * n8 + static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float r = rho_of_hu(hu[i]);
        rho[i] = r;
        const int m = (r >= t0) + (r >= t1) + (r >= t2);
        lmax[m] = max(lmax[m], __float_as_uint(r));
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        unsigned int v = lmax[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(kFull, v, o));
        if ((threadIdx.x & 31) == 0 && v) atomicMax(&s_max[m], v);
    }
    __syncthreads();
    if (threadIdx.x < 4 && s_max[threadIdx.x]) atomicMax(&rho_max_bits[threadIdx.x], s_max[threadIdx.x]);
    if (blockIdx.x == 0 && threadIdx.x == 0) { thr[0] = t0; thr[1] = t1; thr[2] = t2; }
}

// ------------------------------------------ radiological thickness ----
// Radiological thickness (Sec. 2.2, item 1): t = sum_v rho_v l_v along the
// ray from the source to each pixel centre on the sensitive layer's
// mid-plane.  Incremental voxel traversal (the Siddon parametrisation walked
// plane by plane); crossings in single precision relative to the source,
// products accumulated in double.
__global__ void k_tmap(TmapArgs A, double* __restrict__ t) {
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= A.npx * A.npy) return;
    const int ix = pix % A.npx, iy = pix / A.npx;
    const float X = -A.hwx + (ix + 0.5f) * A.pitch, Y = -A.hwy + (iy + 0.5f) * A.pitch, Z = A.zs;
    float d[3], S[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        S[k] = A.src[k];
        d[k] = A.iso[k] + X * A.ex[k] + Y * A.ey[k] + Z * A.ez[k] - S[k];
    }
    const float len = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const int n[3] = {A.nx, A.ny, A.nz};
    const float o[3] = {A.ox, A.oy, A.oz}, v[3] = {A.vx, A.vy, A.vz};
    float amin = 0.0f, amax = 1.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = o[k], hi = o[k] + n[k] * v[k];
        if (d[k] != 0.0f) {
            const float a0 = (lo - S[k]) / d[k], a1 = (hi - S[k]) / d[k];
            amin = fmaxf(amin, fminf(a0, a1));
            amax = fminf(amax, fmaxf(a0, a1));
        } else if (S[k] <= lo || S[k] >= hi) {
            amax = -1.0f;
        }
    }
    double acc = 0.0;
    if (amin < amax) {
        int idx[3], stp[3], plane[3];
        float anext[3], inv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float pk = S[k] + amin * d[k];
            idx[k] = min(max(__float2int_rd((pk - o[k]) / v[k]), 0), n[k] - 1);
            stp[k] = (d[k] > 0.0f) ? 1 : (d[k] < 0.0f ? -1 : 0);
            plane[k] = idx[k] + (stp[k] > 0 ? 1 : 0);
            inv[k] = (stp[k] != 0) ? 1.0f / d[k] : 0.0f;
            anext[k] = (stp[k] != 0) ? (o[k] + plane[k] * v[k] - S[k]) * inv[k] : INFINITY;
        }
        float acur = amin;
        const int maxit = n[0] + n[1] + n[2] + 3;
        for (int it = 0; it < maxit; ++it) {
            int k = 0;
            if (anext[1] < anext[k]) k = 1;
            if (anext[2] < anext[k]) k = 2;
            const float aend = fminf(anext[k], amax);
            const float rho = __ldg(&A.rho[(static_cast<size_t>(idx[2]) * A.ny + idx[1]) * A.nx + idx[0]]);
            // the segment's product in single precision, the sum in double
            acc += static_cast<double>(rho * ((aend - acur) * len));
            if (anext[k] >= amax) break;
            acur = anext[k];
            idx[k] += stp[k];
            if (idx[k] < 0 || idx[k] >= n[k]) break;
            plane[k] += stp[k];
            anext[k] = (o[k] + plane[k] * v[k] - S[k]) * inv[k];
        }
    }
    t[pix] = acc + A.t_offset;
}

// ------------------------------------------------ dose statistics ----
// Per pixel: dose per history D = sum_b E_b / N, batch doses D_b = E_b / N_b,
// sigma = sqrt(sum_b (D_b - D)^2 / (B (B - 1))).  Also the image maximum.
__global__ void k_dose(const unsigned long long* __restrict__ tally, int npix, int B, const double* __restrict__ nb,
                       double n_hist, double conv, double* __restrict__ dose, double* __restrict__ sigma,
                       unsigned long long* max_bits) {
    // per-batch factor from tally units to dose per history, once per block
    __shared__ double s_w[1024];
    __shared__ unsigned long long s_max[32];
    const double per_q = 1.0 / 2.56e8;              // MeV per tally unit
    for (int b = threadIdx.x; b < B; b += blockDim.x) s_w[b] = per_q / nb[b] * conv;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double dm = 0.0;
    if (i < npix) {
        double sum = 0.0;
        for (int b = 0; b < B; ++b) sum += static_cast<double>(tally[static_cast<size_t>(b) * npix + i]);
        dm = sum * per_q / n_hist * conv;
        double ss = 0.0;
        for (int b = 0; b < B; ++b) {
            const double db = static_cast<double>(tally[static_cast<size_t>(b) * npix + i]) * s_w[b];
            ss += (db - dm) * (db - dm);
        }
        dose[i] = dm;
        if (sigma) sigma[i] = sqrt(ss / (static_cast<double>(B) * (B - 1)));
    }
    // block maximum (doses are >= 0, so their bit patterns order like the values), one atomic per block
    unsigned long long bits = __double_as_longlong(dm);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_down_sync(kFull, bits, o);
        bits = ob > bits ? ob : bits;
    }
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = bits;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) m = s_max[w] > m ? s_max[w] : m;
        if (m) atomicMax(max_bits, m);
    }
}

// Mean relative uncertainty over pixels above half the maximum: per-block
// partial sums (fixed order), then a single-block final sum.
__global__ void k_u_partial(const double* __restrict__ dose, const double* __restrict__ sigma, int npix,
                            const unsigned long long* max_bits, double* part_sum, unsigned int* part_cnt) {
    __shared__ double s_sum[256];
    __shared__ unsigned int s_cnt[256];
    const double half = 0.5 * __longlong_as_double(static_cast<long long>(*max_bits));
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    unsigned int c = 0u;
    if (i < npix && dose[i] > half) { v = sigma[i] / dose[i]; c = 1u; }
    s_sum[threadIdx.x] = v;
    s_cnt[threadIdx.x] = c;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) { s_sum[threadIdx.x] += s_sum[threadIdx.x + s]; s_cnt[threadIdx.x] += s_cnt[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part_sum[blockIdx.x] = s_sum[0]; part_cnt[blockIdx.x] = s_cnt[0]; }
}

__global__ void k_u_final(const double* part_sum, const unsigned int* part_cnt, int nparts, double* u) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        unsigned long long c = 0ull;
        for (int i = 0; i < nparts; ++i) { s += part_sum[i]; c += part_cnt[i]; }
        *u = c ? s / static_cast<double>(c) : __longlong_as_double(0x7ff8000000000000ll);
    }
}

// ------------------------------------------------- k(t, s) table ----
// signal = k_scale * k(t, s) * dose.  ks holds the table's column already
// interpolated at the field's s (the bilinear rule taken one axis at a time);
// here the per-pixel linear step along t, clamped at the end nodes.
__global__ void k_lut(const double* __restrict__ dose, const double* __restrict__ t, int npix,
                      const double* __restrict__ tn, const double* __restrict__ ks, int nt, double k_scale,
                      float* __restrict__ signal) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix) return;
    double tt = fmin(fmax(t[i], tn[0]), tn[nt - 1]);
    int lo = 0, hi = nt - 1;                       // largest node index with tn <= tt
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tn[mid] <= tt) lo = mid; else hi = mid;
    }
    lo = min(lo, nt - 2);
    const double f = (tt - tn[lo]) / (tn[lo + 1] - tn[lo]);
    const double k = ks[lo] + f * (ks[lo + 1] - ks[lo]);
    signal[i] = static_cast<float>(k_scale * k * dose[i]);
}

// ---------------------------------------------------------- diagnostics --
__global__ void k_test_philox(const uint32_t* in, uint32_t* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox4x32_10(make_uint4(in[6 * i], in[6 * i + 1], in[6 * i + 2], in[6 * i + 3]), in[6 * i + 4],
                                  in[6 * i + 5]);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

__global__ void k_test_uniforms(unsigned long long seed, unsigned long long hist, uint32_t ord, int n, float* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const PhiloxKey K = philox_key(seed);
    Rng r;
    r.setup(K, hist, ord, 0u);
    for (int i = 0; i < n; ++i) out[i] = r.u(K);
}

// ----------------------------------------------------------- launchers ---
cudaError_t launch_hu_to_rho(const int16_t* hu, float* rho, size_t n, unsigned int* rho_max_bits, float* thr,
                             int sm_count, cudaStream_t s) {
    const int block = 256;
    size_t want = (n / 8 + block - 1) / block;
    int grid = static_cast<int>(want < static_cast<size_t>(sm_count) * 8 ? want : static_cast<size_t>(sm_count) * 8);
    if (grid < 1) grid = 1;
    k_hu_to_rho<<<grid, block, 0, s>>>(hu, rho, n, rho_max_bits, thr);
    return cudaGetLastError();
}

// One axis of the box extremes behind the homogeneity flags: for each voxel
// the least and greatest value over `radius` voxels either side along `axis`
// (cut at the CT's edge), packed as (least & 0xffff) | (greatest << 16).  The
// first pass reads the clamped HU itself; the last turns the box extremes
// into the flag, written as the sign of the voxel's density.  Extremes of a box are the extremes of its rows' extremes,
// and materials rise with HU, so one material means that the least and the
// greatest value have the same material.
__device__ __forceinline__ int clamp_hu_dev(int h) { return min(max(h, -1024), 3071); }
__device__ __forceinline__ int material_of_hu(int h) { return (h < -900) ? 0 : (h < -200) ? 1 : (h < 300) ? 2 : 3; }

__global__ void k_hom_pass(const int16_t* __restrict__ hu, const int* __restrict__ in, int nx, int ny, int nz,
                           int axis, int radius, int span, int* __restrict__ out, const float* __restrict__ rho,
                           float* __restrict__ rho_hom) {
    const size_t n = static_cast<size_t>(nx) * ny * nz;
    const int dim = (axis == 0) ? nx : (axis == 1) ? ny : nz;
    const size_t stride = (axis == 0) ? 1 : (axis == 1) ? static_cast<size_t>(nx) : static_cast<size_t>(nx) * ny;
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < n;
         v += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int ix = static_cast<int>(v % nx), iy = static_cast<int>((v / nx) % ny), iz = static_cast<int>(v / (static_cast<size_t>(nx) * ny));
        const int k = (axis == 0) ? ix : (axis == 1) ? iy : iz;
        int lo = 1 << 20, hi = -(1 << 20);
        for (int d = -radius; d <= radius; ++d) {
            if (k + d < 0 || k + d >= dim) continue;
            const size_t w = v + static_cast<ptrdiff_t>(d) * static_cast<ptrdiff_t>(stride);
            int a, b;
            if (hu) {
                a = b = clamp_hu_dev(__ldg(&hu[w]));
            } else {
                const int q = __ldg(&in[w]);
                a = static_cast<int16_t>(q & 0xffff);
                b = q >> 16;
            }
            lo = min(lo, a);
            hi = max(hi, b);
        }
        if (rho_hom) {
            const bool inside = ix >= radius && ix < nx - radius && iy >= radius && iy < ny - radius &&
                                iz >= radius && iz < nz - radius;
            const bool hom = inside && material_of_hu(lo) == material_of_hu(hi) && hi - lo <= span;
            rho_hom[v] = __int_as_float(__float_as_int(__ldg(&rho[v])) | (hom ? 0x80000000 : 0));
        } else {
            out[v] = (lo & 0xffff) | (hi << 16);
        }
    }
}

cudaError_t launch_homogeneity(const int16_t* hu, const float* rho, int nx, int ny, int nz, int radius, int span,
                               int* tmp, float* rho_hom, int sm_count, cudaStream_t s) {
    const size_t n = static_cast<size_t>(nx) * ny * nz;
    int* a = tmp;
    int* b = tmp + n;
    const int grid = sm_count * 8, block = 256;
    k_hom_pass<<<grid, block, 0, s>>>(hu, nullptr, nx, ny, nz, 0, radius, span, a, nullptr, nullptr);
    k_hom_pass<<<grid, block, 0, s>>>(nullptr, a, nx, ny, nz, 1, radius, span, b, nullptr, nullptr);
    k_hom_pass<<<grid, block, 0, s>>>(nullptr, b, nx, ny, nz, 2, radius, span, nullptr, rho, rho_hom);
    return cudaGetLastError();
}

cudaError_t launch_macro_grid(const float* rho, int nx, int ny, int nz, int M, int mgx, int mgy, int mgz,
                              float thr_bone, float2* grid, int sm_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(grid, 0, sizeof(float2) * static_cast<size_t>(mgx) * mgy * mgz, s);
    if (e != cudaSuccess) return e;
    k_macro_grid<<<sm_count * 8, 256, 0, s>>>(rho, nx, ny, nz, M, mgx, mgy, thr_bone,
                                              reinterpret_cast<unsigned int*>(grid));
    return cudaGetLastError();
}

cudaError_t launch_tmap(const TmapArgs& A, double* t, cudaStream_t s) {
    const int npix = A.npx * A.npy, block = 128;
    k_tmap<<<(npix + block - 1) / block, block, 0, s>>>(A, t);
    return cudaGetLastError();
}

__global__ void k_batch_counts(double* nb, int B, unsigned long long n) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) nb[b] = static_cast<double>(n / B + (static_cast<unsigned long long>(b) < n % B ? 1ull : 0ull));
}

// Source fluence on the EPID grid (Sec. 2.1.1: the MLC-modulated source the
// transport samples).  Rectangle i of a field carries probability
// cdf[i] - cdf[i-1] spread uniformly over its area; a pixel takes the density
// of the rectangle (one per segment) that holds its centre projected to the
// isocentre plane.  Rectangles are half-open [x0, x1) x [y0, y1) and
// neighbours share their float edges, so the pixel ranges below, computed
// from those edges, tile without gaps or overlaps.  One block per rectangle,
// one double atomic per covered pixel.
__global__ void k_fluence(const float4* __restrict__ rect, const double* __restrict__ cdf, int npx, int npy,
                          double pitch, double mag, double* __restrict__ F) {
    const int i = blockIdx.x;
    const float4 r = rect[i];
    const double w = cdf[i] - (i > 0 ? cdf[i - 1] : 0.0);
    const double area = (static_cast<double>(r.y) - r.x) * (static_cast<double>(r.w) - r.z);
    if (!(w > 0.0) || !(area > 0.0)) return;
    const double dens = w / area;
    // first pixel index whose centre (-n p / 2 + (k + 1/2) p) / mag is >= the edge
    auto first = [&](double edge, int n) {
        const double k = ceil((edge * mag + 0.5 * n * pitch) / pitch - 0.5);
        return static_cast<int>(fmin(fmax(k, 0.0), static_cast<double>(n)));
    };
    const int ix0 = first(r.x, npx), ix1 = first(r.y, npx);
    const int iy0 = first(r.z, npy), iy1 = first(r.w, npy);
    const int wx = ix1 - ix0, hy = iy1 - iy0;
    if (wx <= 0 || hy <= 0) return;
    const long long n = static_cast<long long>(wx) * hy;
    for (long long q = threadIdx.x; q < n; q += blockDim.x) {
        const int yy = static_cast<int>(q / wx), xx = static_cast<int>(q - static_cast<long long>(yy) * wx);
        atomicAdd(F + static_cast<size_t>(iy0 + yy) * npx + ix0 + xx, dens);
    }
}

cudaError_t launch_fluence(const float4* rect, const double* cdf, int n_rect, int npx, int npy, double pitch,
                           double mag, double* F, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(F, 0, sizeof(double) * static_cast<size_t>(npx) * npy, s);
    if (e != cudaSuccess || n_rect <= 0) return e;
    k_fluence<<<n_rect, 256, 0, s>>>(rect, cdf, npx, npy, pitch, mag, F);
    return cudaGetLastError();
}

// Region statistics (Sec. 2.2 calibration region, Sec. 2.3 uncertainty): per
// batch b the exact integer sum of its sub-tally over pixels [ix0, ix0 + w) x
// [iy0, iy0 + h); then, one thread, the region's mean dose per history
// D = sum_b E_b / (N n_pix) and the batch standard error of the region mean,
// sqrt(sum_b (D_b - D)^2 / (B (B - 1))) with D_b = E_b / (N_b n_pix).
__global__ void k_region_sums(const unsigned long long* __restrict__ tally, int npx, int npix, int ix0, int iy0,
                              int w, int h, unsigned long long* __restrict__ sums) {
    const int b = blockIdx.y;
    const long long n = static_cast<long long>(w) * h;
    const unsigned long long* t = tally + static_cast<size_t>(b) * npix;
    unsigned long long acc = 0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(i / w), q = static_cast<int>(i - static_cast<long long>(r) * w);
        acc += t[static_cast<size_t>(iy0 + r) * npx + ix0 + q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sums + b, acc);
}

__global__ void k_region_stats(const unsigned long long* __restrict__ sums, const double* __restrict__ nb, int B,
                               double n_hist, double conv_per_pix, double* __restrict__ out) {
    const double per_q = 1.0 / 2.56e8;              // MeV per tally unit
    double tot = 0.0;
    for (int b = 0; b < B; ++b) tot += static_cast<double>(sums[b]);
    const double mean = tot * per_q / n_hist * conv_per_pix;
    double ss = 0.0;
    for (int b = 0; b < B; ++b) {
        const double db = static_cast<double>(sums[b]) * per_q / nb[b] * conv_per_pix;
        ss += (db - mean) * (db - mean);
    }
    out[0] = mean;
    out[1] = sqrt(ss / (static_cast<double>(B) * (B - 1)));
}

cudaError_t launch_region_stats(const unsigned long long* tally, int npx, int npy, int B, const double* nb,
                                double n_hist, double conv, int ix0, int ix1, int iy0, int iy1,
                                unsigned long long* sums, double* out, cudaStream_t s) {
    const int w = ix1 - ix0, h = iy1 - iy0;
    const long long n = static_cast<long long>(w) * h;
    cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * B, s);
    if (e != cudaSuccess) return e;
    const int block = 256;
    const int gx = static_cast<int>(std::min<long long>((n + block - 1) / block, 64));
    k_region_sums<<<dim3(gx, B), block, 0, s>>>(tally, npx, npx * npy, ix0, iy0, w, h, sums);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_region_stats<<<1, 1, 0, s>>>(sums, nb, B, n_hist, conv / static_cast<double>(n), out);
    return cudaGetLastError();
}

cudaError_t launch_batch_counts(double* nb, int B, unsigned long long n, cudaStream_t s) {
    k_batch_counts<<<(B + 127) / 128, 128, 0, s>>>(nb, B, n);
    return cudaGetLastError();
}

cudaError_t launch_dose(const unsigned long long* tally, int npix, int B, const double* nb, double n_hist,
                        double conv, double* dose, double* sigma, unsigned long long* max_bits, double* part_sum,
                        unsigned int* part_cnt, double* u, cudaStream_t s) {
    const int block = 256, grid = (npix + block - 1) / block;
    cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_dose<<<grid, block, 0, s>>>(tally, npix, B, nb, n_hist, conv, dose, sigma, max_bits);
    if (u && sigma) {
        k_u_partial<<<grid, block, 0, s>>>(dose, sigma, npix, max_bits, part_sum, part_cnt);
        k_u_final<<<1, 32, 0, s>>>(part_sum, part_cnt, grid, u);
    }
    return cudaGetLastError();
}

// Global gamma index (Low et al. 1998) of `ev` against `ref`, one thread per
// reference pixel: above the low-dose threshold, the least
// sqrt(r^2 / dta^2 + (ev(x + r) - ref(x))^2 / dd^2) over sub-grid offsets r
// of step h within the search radius, ev bilinearly interpolated (clamped at
// the border); dd = dd_frac * max(ref).  FP64 throughout.
__device__ double bilin_clamped(const double* img, int nx, int ny, double fx, double fy) {
    fx = fmin(fmax(fx, 0.0), static_cast<double>(nx - 1));
    fy = fmin(fmax(fy, 0.0), static_cast<double>(ny - 1));
    const int x0 = static_cast<int>(floor(fx)), y0 = static_cast<int>(floor(fy));
    const int x1 = x0 + 1 < nx ? x0 + 1 : x0, y1 = y0 + 1 < ny ? y0 + 1 : y0;
    const double ax = fx - x0, ay = fy - y0;
    return (1 - ay) * ((1 - ax) * img[static_cast<size_t>(y0) * nx + x0] + ax * img[static_cast<size_t>(y0) * nx + x1]) +
           ay * ((1 - ax) * img[static_cast<size_t>(y1) * nx + x0] + ax * img[static_cast<size_t>(y1) * nx + x1]);
}

__global__ void k_max_f64(const double* __restrict__ a, size_t n, unsigned long long* max_bits) {
    double m = 0.0;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        m = fmax(m, a[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(max_bits, static_cast<unsigned long long>(__double_as_longlong(m)));
}

__global__ void k_gamma(const double* __restrict__ ref, const double* __restrict__ ev, int nx, int ny, double pix,
                        double dd_frac, double dta, double thr_frac, double h, double rad,
                        const unsigned long long* max_bits, double* gam, unsigned long long* counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny) return;
    const double rmax = __longlong_as_double(static_cast<long long>(*max_bits));
    const double ddabs = dd_frac * rmax;
    const int x = i % nx, y = i / nx;
    if (ref[i] < thr_frac * rmax) {
        if (gam) gam[i] = nan("");
        return;
    }
    const int nsub = static_cast<int>(ceil(rad / h));
    double best = INFINITY;
    for (int sy = -nsub; sy <= nsub && best > 0.0; ++sy) {
        for (int sx = -nsub; sx <= nsub; ++sx) {
            const double dx = sx * h, dy = sy * h;
            const double r2 = dx * dx + dy * dy;
            if (r2 > rad * rad) continue;
            const double dist2 = r2 / (dta * dta);
            if (dist2 >= best) continue;
            const double v = bilin_clamped(ev, nx, ny, x + dx / pix, y + dy / pix);
            const double dv = (v - ref[i]) / ddabs;
            const double g2 = dist2 + dv * dv;
            if (g2 < best) best = g2;
        }
    }
    const double gv = sqrt(best);
    if (gam) gam[i] = gv;
    atomicAdd(&counts[0], 1ull);
    if (gv <= 1.0) atomicAdd(&counts[1], 1ull);
}

__device__ double bilin_clamped(const double* img, int nx, int ny, double fx, double fy);

// Plan image: acc_dose += w dose, acc_signal += w k(t, s) dose (FP64 sums
// over the fields of a batch).
__global__ void k_plan_accum(const double* __restrict__ dose, const double* __restrict__ t, int npix,
                             const double* __restrict__ tn, const double* __restrict__ ks, int nt, double k_scale,
                             double w, double* __restrict__ acc_dose, double* __restrict__ acc_signal) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix) return;
    acc_dose[i] += w * dose[i];
    if (!acc_signal) return;
    double tt = fmin(fmax(t[i], tn[0]), tn[nt - 1]);
    int lo = 0, hi = nt - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tn[mid] <= tt) lo = mid; else hi = mid;
    }
    lo = min(lo, nt - 2);
    const double f = (tt - tn[lo]) / (tn[lo + 1] - tn[lo]);
    acc_signal[i] += w * k_scale * (ks[lo] + f * (ks[lo + 1] - ks[lo])) * dose[i];
}

cudaError_t launch_plan_accum(const double* dose, const double* t, int npix, const double* tn, const double* ks,
                              int nt, double k_scale, double w, double* acc_dose, double* acc_signal,
                              cudaStream_t s) {
    k_plan_accum<<<(npix + 255) / 256, 256, 0, s>>>(dose, t, npix, tn, ks, nt, k_scale, w, acc_dose, acc_signal);
    return cudaGetLastError();
}

// Bilinear resampling between two pixel grids centred on the same axis
// (pixel centres at ((i + 0.5) - n / 2) pitch), clamped at the border.
__global__ void k_resample(const double* __restrict__ src, int snx, int sny, double sp, double* __restrict__ dst,
                           int dnx, int dny, double dp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dnx * dny) return;
    const int x = i % dnx, y = i / dnx;
    const double X = ((x + 0.5) - 0.5 * dnx) * dp, Y = ((y + 0.5) - 0.5 * dny) * dp;
    dst[i] = bilin_clamped(src, snx, sny, X / sp + 0.5 * snx - 0.5, Y / sp + 0.5 * sny - 0.5);
}

cudaError_t launch_resample(const double* src, int snx, int sny, double sp, double* dst, int dnx, int dny, double dp,
                            cudaStream_t s) {
    const int n = dnx * dny;
    k_resample<<<(n + 255) / 256, 256, 0, s>>>(src, snx, sny, sp, dst, dnx, dny, dp);
    return cudaGetLastError();
}

__global__ void k_vox_dose(const unsigned long long* __restrict__ vox, const float* __restrict__ rho, size_t n,
                           double conv, double* __restrict__ dose) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        dose[i] = static_cast<double>(vox[i]) * conv / static_cast<double>(rho[i]);
}

cudaError_t launch_vox_dose(const unsigned long long* vox, const float* rho, size_t n, double conv, double* dose,
                            cudaStream_t s) {
    k_vox_dose<<<static_cast<unsigned>(std::min<size_t>((n + 255) / 256, 148 * 32)), 256, 0, s>>>(vox, rho, n, conv,
                                                                                                  dose);
    return cudaGetLastError();
}

cudaError_t launch_gamma(const double* ref, const double* ev, int nx, int ny, double pix, double dd_frac, double dta,
                         double thr_frac, double h, double rad, double* gam, unsigned long long* scratch,
                         cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const size_t n = static_cast<size_t>(nx) * ny;
    k_max_f64<<<static_cast<unsigned>(std::min<size_t>((n + 255) / 256, 1184)), 256, 0, s>>>(ref, n, scratch);
    k_gamma<<<static_cast<unsigned>((n + 127) / 128), 128, 0, s>>>(ref, ev, nx, ny, pix, dd_frac, dta, thr_frac, h,
                                                                   rad, scratch, gam, scratch + 1);
    return cudaGetLastError();
}

cudaError_t launch_lut(const double* dose, const double* t, int npix, const double* tn, const double* ks, int nt,
                       double k_scale, float* signal, cudaStream_t s) {
    const int block = 256;
    k_lut<<<(npix + block - 1) / block, block, 0, s>>>(dose, t, npix, tn, ks, nt, k_scale, signal);
    return cudaGetLastError();
}

cudaError_t launch_test_philox(const uint32_t* in, uint32_t* out, int n, cudaStream_t s) {
    k_test_philox<<<(n + 127) / 128, 128, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_test_uniforms(unsigned long long seed, unsigned long long hist, uint32_t ord, int n, float* out,
                                 cudaStream_t s) {
    k_test_uniforms<<<1, 32, 0, s>>>(seed, hist, ord, n, out);
    return cudaGetLastError();
}

}  // namespace mc
