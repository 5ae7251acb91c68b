// Argument blocks and launchers of the denoiser's kernels (internal header).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dn {

// One activation source of a convolution (two for a concatenated input):
// channels stored (a multiple of 8) and the chunk of channels one K step
// loads (16, 32 or 64: the tile row is 32, 64 or 128 bytes).
struct ConvSrc {
    int C, CW, nch;
};

// Implicit-GEMM convolution (forward, or input gradient with transposed
// weights): out[n,y,x,j] = epilogue(sum over taps t, sources s, channels c of
// src_s[n, y+dy_t-p, x+dx_t-p, c] * Wop_s[j][t][c]).
struct ConvArgs {
    int nsrc;
    ConvSrc src[2];
    int k;                      // 1 or 3 (p = k / 2)
    int Nb, H, W;
    int N;                      // output channels (GEMM N)
    int N_tile, tmem_cols;
    int nk;                     // K steps = k*k * (chunks of all sources)
    int stages;
    int grid;                   // persistent CTAs (one per SM)
    // resident-weight variant (rows_per_tile > 0): R output rows per tile,
    // packed weights of source s at byte w_off[s] of a w_bytes region
    int rows_per_tile;
    int dxn;                    // column taps in N (3x3, N <= 64): tiles of 126 pixels
    int epi_groups;             // streamed and column-tap variants: TMEM accumulator buffers, one
                                // epilogue warpgroup each (resident variant: 2)
    int buf_cols;               // TMEM columns per buffer (streamed and column-tap variants)
    uint32_t w_bytes, w_bytes_real, w_off[2];
    uint32_t stage_bytes, a_region;
    uint32_t idesc;             // instruction descriptor of one MMA: M = 128, N = n_slice
    // the N columns of a tile are split into n_issue slices of n_slice, each
    // issued by its own warp: a warp issues one tcgen05.mma per ~170 cycles
    // whatever its N, so narrow tiles need several issuers to keep the tensor
    // core busy
    int n_issue, n_slice;
    const float* bias;          // [N] or null
    int relu;
    int ndst, dst_split;        // channels [0, split) -> dst[0], [split, N) -> dst[1]
    __nv_bfloat16* dst[2];
    int dst_C[2];
    const __nv_bfloat16* mask[2];   // if set: zero where mask <= 0 (same layout as dst)
    unsigned* err;
};

// Convolution kernels (streamed and column-tap): at most 4 accumulator
// buffers, each drained by its own epilogue warpgroup (warps 4 + 4g ..
// 7 + 4g), after the producer and the three MMA warps.
constexpr int kConvMaxGroups = 4;
constexpr int kConvMaxN = 512;      // output channels of one convolution
constexpr int kConvMaxThreads = 32 * (4 + 4 * kConvMaxGroups);
// Column-tap convolution: K steps per tile (3 row taps x channel chunks) at most.
constexpr int kDxnMaxSteps = 24;

// MMA-issuing warps of the weight-gradient kernel (see k_wgrad).
constexpr int kWgradIssuers = 3;

// Weight gradient: dW[co][dy][dx][coff_s + c] += sum over pixels of
// dz[n,y,x,co] * src_s[n, y+dy-p, x+dx-p, c].  mode 0: M = 128 output
// channels; mode 1 (Co = 32 or 64, k = 3): M = G = 128 / Co taps x Co.
struct WgradArgs {
    int Nb, H, W, k;
    int mode, G;
    int Co, co_tiles;
    int nsrc;
    int src_C[2], src_coff[2], src_chunks[2];
    int ci_total;
    int ksteps, splits;
    int stages;
    uint32_t stage_bytes, b_region;
    uint32_t idesc;
    int tmem_cols;
    float* dW;
    unsigned* err;
};

cudaError_t conv_prepare();
cudaError_t launch_conv(const CUtensorMap* ta, const CUtensorMap* tb, const ConvArgs& a, cudaStream_t s);
cudaError_t launch_wgrad(const CUtensorMap* tz, const CUtensorMap* tx, const WgradArgs& a, cudaStream_t s);

// Pointwise and reduction kernels.
cudaError_t launch_maxpool(const __nv_bfloat16* x, __nv_bfloat16* y, int Nb, int H, int W, int C, cudaStream_t s);
cudaError_t launch_maxpool_bwd(const __nv_bfloat16* x, const __nv_bfloat16* dy, const __nv_bfloat16* add,
                               __nv_bfloat16* dx, int Nb, int H, int W, int C, cudaStream_t s);
cudaError_t launch_upsample(const __nv_bfloat16* x, __nv_bfloat16* y, int Nb, int h, int w, int C, cudaStream_t s);
cudaError_t launch_upsample_bwd(const __nv_bfloat16* dy, __nv_bfloat16* dx, int Nb, int h, int w, int C,
                                cudaStream_t s);
cudaError_t launch_bias_grad(const __nv_bfloat16* dz, int Cz, int Co, long long npix, float* db, cudaStream_t s);
cudaError_t launch_mse(const __nv_bfloat16* y, int y_stride, const __nv_bfloat16* t, long long n,
                       __nv_bfloat16* dy, int dy_stride, double* partials, int nparts, double* loss, cudaStream_t s);
int mse_parts();
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t s);
// fp32 master weights [Co][k][k][Ci_total] -> bf16 operand of one source,
// [rows >= Co][k*k][nch*CW] (forward) or the flipped transpose
// [rows >= Ci_total][k*k][nchz*CWz] (input gradient); padding is zero.
cudaError_t launch_pack_fwd(const float* w, int Co, int rows, int k, int ci_total, int coff, int C, int CW, int nch,
                            __nv_bfloat16* out, cudaStream_t s);
cudaError_t launch_pack_dgrad(const float* w, int Co, int k, int ci_total, int rows, int CWz, int nchz,
                              __nv_bfloat16* out, cudaStream_t s);
// Column-taps-in-N operand [(dx, o)][(dy, chunk, c)], o < Nout (3 * Nout rows).
cudaError_t launch_pack_dxn(const float* w, int Co, int ci_total, int coff, int C, int CW, int nch, int dgrad,
                            int Nout, __nv_bfloat16* out, cudaStream_t s);
// Planar float32 [image][planes][hw] -> NHWC bf16 with out_C stored channels
// (channels >= planes zero); plane 0 is multiplied by scale.
cudaError_t launch_prep(const float* img, int planes, long long hw, float scale, long long npix,
                        __nv_bfloat16* out, int out_C, cudaStream_t s);
cudaError_t launch_to_f32(const __nv_bfloat16* x, int stride, long long npix, float scale, float* out,
                          cudaStream_t s);

}  // namespace dn
