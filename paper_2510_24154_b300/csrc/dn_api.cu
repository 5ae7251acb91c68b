// C ABI of the EPID-image denoiser (declared in archer_denoise.h): the U-Net
// runner (buffers, TMA descriptors, forward, backward, Adam) and the
// primitive calls, all on the kernels of dn_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "archer_denoise.h"
#include "dn_kernels.cuh"
#include "dn_tc.cuh"

using bf16 = __nv_bfloat16;
using dn::ConvArgs;
using dn::WgradArgs;

namespace {

// ------------------------------------------------------- TMA descriptors --

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

int cw_for(int C) { return C >= 64 ? 64 : (C > 16 ? 32 : 16); }
int chunks(int C, int CW) { return (C + CW - 1) / CW; }

CUtensorMapSwizzle tma_swizzle(int CW) {
    return CW == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CW == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}

// NHWC bf16 activation, box = (box_c channels) x (128 pixels of one row).
bool act_map(CUtensorMap* m, const void* base, int Nb, int H, int W, int C, int box_c) {
    EncodeTiledFn f = encoder();
    if (!f) return false;
    const cuuint64_t dims[4] = {static_cast<cuuint64_t>(C), static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H),
                                static_cast<cuuint64_t>(Nb)};
    const cuuint64_t strides[3] = {static_cast<cuuint64_t>(C) * 2, static_cast<cuuint64_t>(W) * C * 2,
                                   static_cast<cuuint64_t>(H) * W * C * 2};
    const cuuint32_t box[4] = {static_cast<cuuint32_t>(box_c), 128, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, tma_swizzle(box_c), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row-major bf16 matrix [rows][cols] (K-major operand), box = box_r rows x box_c columns.
bool mat_map(CUtensorMap* m, const void* base, int rows, int cols, int box_c, int box_r) {
    EncodeTiledFn f = encoder();
    if (!f) return false;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * 2};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_c), static_cast<cuuint32_t>(box_r)};
    const cuuint32_t es[2] = {1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, tma_swizzle(box_c), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

uint32_t pow2_at_least(uint32_t v) {
    uint32_t p = 32;
    while (p < v) p <<= 1;
    return p;
}

// ------------------------------------------------------------ planning ----

// Output tiling of a GEMM with N columns: at most 256 per tile.
void n_tiling(int N, int& n_tile, int& n_tiles) {
    n_tiles = (N + 255) / 256;
    const int per = (N + n_tiles - 1) / n_tiles;
    n_tile = ((per + 15) / 16) * 16;
}

struct ConvPlan {
    ConvArgs a{};
    CUtensorMap ta[2], tb[2];
};

// A convolution launch (forward or input gradient).  src/srcC: activation
// sources; wop[s]: packed bf16 operand [wrows][k*k*nch_s*CW_s].
// Column-taps-in-N variant: 3x3, 32 or 64 output channels, resident weights.
bool dxn_fits(int k, int N, int nsrc, const int srcC[2]) {
    if (k != 3 || !(N == 32 || N == 64)) return false;
    size_t bytes = 0;
    int steps = 0;
    for (int s = 0; s < nsrc; ++s) {
        const int CW = cw_for(srcC[s]);
        bytes = (bytes + 1023) / 1024 * 1024 + static_cast<size_t>(3 * chunks(srcC[s], CW)) * 3 * N * CW * 2;
        steps += 3 * chunks(srcC[s], CW);
    }
    return bytes <= 150u * 1024u && steps <= dn::kDxnMaxSteps;
}

bool plan_conv(ConvPlan& P, int nsrc, const bf16* const src[2], const int srcC[2], int Nb, int H, int W, int k,
               const bf16* const wop[2], int wrows, int N, const float* bias, int relu, int ndst, int split,
               bf16* const dst[2], const int dstC[2], const bf16* const mask[2], unsigned* err, int sm_count,
               bool resident_ok = true, bool dxn = false) {
    ConvArgs& a = P.a;
    std::memset(&a, 0, sizeof(a));
    a.nsrc = nsrc;
    a.k = k;
    a.Nb = Nb; a.H = H; a.W = W;
    a.N = N;
    if (N < 1 || N > dn::kConvMaxN) return false;
    int n_tiles;
    n_tiling(N, a.N_tile, n_tiles);
    a.tmem_cols = static_cast<int>(pow2_at_least(static_cast<uint32_t>(a.N_tile)));
    int cwmax = 16, nch_total = 0;
    for (int s = 0; s < nsrc; ++s) {
        a.src[s].C = srcC[s];
        a.src[s].CW = cw_for(srcC[s]);
        a.src[s].nch = chunks(srcC[s], a.src[s].CW);
        cwmax = std::max(cwmax, a.src[s].CW);
        nch_total += a.src[s].nch;
        if (!act_map(&P.ta[s], src[s], Nb, H, W, srcC[s], a.src[s].CW)) return false;
        if (dxn) {
            if (!mat_map(&P.tb[s], wop[s], 3 * N, 3 * a.src[s].nch * a.src[s].CW, a.src[s].CW, 3 * N)) return false;
        } else if (!mat_map(&P.tb[s], wop[s], wrows, k * k * a.src[s].nch * a.src[s].CW, a.src[s].CW, a.N_tile)) {
            return false;
        }
    }
    if (nsrc == 1) {
        P.ta[1] = P.ta[0];
        P.tb[1] = P.tb[0];
    }
    a.nk = k * k * nch_total;
    a.a_region = 128u * cwmax * 2u;
    const uint32_t b_bytes = ((static_cast<uint32_t>(a.N_tile) * cwmax * 2u + 1023u) / 1024u) * 1024u;
    a.stage_bytes = a.a_region + b_bytes;
    a.stages = std::max(2, std::min(16, static_cast<int>((200u * 1024u) / a.stage_bytes)));
    a.grid = sm_count;
    // resident weights when they fit: R output rows per tile (TMEM holds two
    // sets of R accumulators of N_tile columns)
    uint32_t wb = 0, w_off1 = 0;
    for (int s = 0; s < nsrc; ++s) {
        if (s == 1) {
            wb = (wb + 1023u) / 1024u * 1024u;
            w_off1 = wb;
        }
        wb += static_cast<uint32_t>(k * k * a.src[s].nch) * a.N_tile * a.src[s].CW * 2u;
    }
    const uint32_t w_region = (wb + 1023u) / 1024u * 1024u;
    if (dxn) {
        uint32_t wbx = 0, off1 = 0;
        for (int s = 0; s < nsrc; ++s) {
            if (s == 1) {
                wbx = (wbx + 1023u) / 1024u * 1024u;
                off1 = wbx;
            }
            wbx += static_cast<uint32_t>(3 * a.src[s].nch) * 3u * N * a.src[s].CW * 2u;
        }
        a.dxn = 1;
        a.rows_per_tile = 0;
        a.w_off[0] = 0;
        a.w_off[1] = off1;
        a.w_bytes_real = wbx;
        a.w_bytes = (wbx + 1023u) / 1024u * 1024u;
        a.stage_bytes = a.a_region;
        a.stages = std::max(2, std::min(16, static_cast<int>((205u * 1024u - a.w_bytes) / a.stage_bytes)));
        a.N_tile = N;
        // as many accumulator buffers (each with its own epilogue warpgroup)
        // as TMEM holds: 4 of 128 columns for N = 32, 2 of 256 for N = 64
        a.buf_cols = static_cast<int>(pow2_at_least(static_cast<uint32_t>(3 * N)));
        a.epi_groups = std::min(dn::kConvMaxGroups, 512 / a.buf_cols);
        a.tmem_cols = a.epi_groups * a.buf_cols;
    } else if (n_tiles == 1 && w_region <= 150u * 1024u && resident_ok) {
        // rows per tile first (input reuse), then as many accumulator buffers
        // (epilogue warpgroups) of R rows as TMEM holds, at least two
        int R = 4;
        while (R > 1 && (2 * R * a.N_tile > 512 || R > H)) R >>= 1;
        a.epi_groups = (4 * R * a.N_tile <= 512) ? 4 : 2;
        a.rows_per_tile = R;
        a.w_off[0] = 0;
        a.w_off[1] = w_off1;
        a.w_bytes_real = wb;
        a.w_bytes = w_region;
        a.stage_bytes = a.a_region;
        a.stages = std::max(2, std::min(16, static_cast<int>((205u * 1024u - w_region) / a.stage_bytes)));
        a.tmem_cols = static_cast<int>(pow2_at_least(static_cast<uint32_t>(a.epi_groups * R * a.N_tile)));
    } else {
        a.rows_per_tile = 0;
        a.buf_cols = static_cast<int>(pow2_at_least(static_cast<uint32_t>(a.N_tile)));
        a.epi_groups = std::min(dn::kConvMaxGroups, 512 / a.buf_cols);
        a.tmem_cols = a.epi_groups * a.buf_cols;
    }
    // column slices, one MMA warp each (up to three): a multiple of 16 wide
    if (a.dxn) {
        a.n_issue = 3;                          // one column tap per warp
        a.n_slice = N;
    } else {
        a.n_issue = (a.N_tile % 48 == 0) ? 3 : (a.N_tile % 32 == 0) ? 2 : 1;
        a.n_slice = a.N_tile / a.n_issue;
    }
    a.idesc = dn::idesc_bf16(128, static_cast<uint32_t>(a.n_slice), 0, 0);
    a.bias = bias;
    a.relu = relu;
    a.ndst = ndst;
    a.dst_split = split;
    for (int d = 0; d < ndst; ++d) {
        a.dst[d] = dst[d];
        a.dst_C[d] = dstC[d];
        a.mask[d] = mask ? mask[d] : nullptr;
    }
    a.err = err;
    return true;
}

constexpr int kWgradMinSteps = 32;

struct WgradPlan {
    WgradArgs a{};
    CUtensorMap tz, tx[2];
};

bool plan_wgrad(WgradPlan& P, const bf16* dz, int Cz, int Co, int nsrc, const bf16* const src[2], const int srcC[2],
                int Nb, int H, int W, int k, float* dW, unsigned* err, int sm_count) {
    WgradArgs& a = P.a;
    std::memset(&a, 0, sizeof(a));
    a.Nb = Nb; a.H = H; a.W = W; a.k = k;
    a.Co = Co;
    a.co_tiles = (Co + 127) / 128;
    // narrow layers put several taps into the 128 GEMM rows (dz must hold
    // exactly Co channels so that one box is one tap)
    a.mode = (k == 3 && (Co == 32 || Co == 64) && Cz == Co) ? 1 : 0;
    a.G = a.mode ? 128 / Co : 1;
    a.nsrc = nsrc;
    int coff = 0, nch = 0;
    for (int s = 0; s < nsrc; ++s) {
        a.src_C[s] = srcC[s];
        a.src_coff[s] = coff;
        a.src_chunks[s] = chunks(srcC[s], 64);
        coff += srcC[s];
        nch += a.src_chunks[s];
        if (!act_map(&P.tx[s], src[s], Nb, H, W, srcC[s], 64)) return false;
    }
    if (nsrc == 1) P.tx[1] = P.tx[0];
    if (!act_map(&P.tz, dz, Nb, H, W, Cz, a.mode ? Co : 64)) return false;
    a.ci_total = coff;
    a.ksteps = Nb * H * ((W + 127) / 128);
    const int rows = a.mode == 0 ? a.co_tiles * k : (k * k + a.G - 1) / a.G;
    const int base = rows * nch;
    // K (pixel rows) is split over CTAs to fill the GPU, but each CTA keeps at
    // least kWgradMinSteps K steps: every split adds a full set of f32 atomics
    // to the epilogue (measured: 13.80 -> 13.62 ms per training step)
    int splits = (2 * sm_count + base - 1) / base;
    splits = std::max(1, std::min(splits, a.ksteps / kWgradMinSteps));
    a.splits = splits;
    if (a.mode == 0) {
        a.b_region = 32768u;
        a.stage_bytes = 32768u + static_cast<uint32_t>(k) * 16384u;
        a.idesc = dn::idesc_bf16(128, 64, 1, 1);
    } else {
        a.b_region = static_cast<uint32_t>(a.G) * 128u * Co * 2u;     // G dz boxes = 32 KB
        a.stage_bytes = a.b_region + 16384u;
        a.idesc = dn::idesc_bf16(128, 64, 1, 1);
    }
    // one 64-column accumulator per MMA warp: a column tap each, or a share of the K slices
    a.tmem_cols = static_cast<int>(pow2_at_least(static_cast<uint32_t>(dn::kWgradIssuers * 64)));
    // narrow layers (mode 1): two CTAs per SM of two stages each, so one CTA's
    // start-up and epilogue overlap the other's main loop
    const uint32_t budget = a.mode ? 100u * 1024u : 200u * 1024u;
    a.stages = std::max(2, std::min(6, static_cast<int>(budget / a.stage_bytes)));
    a.dW = dW;
    a.err = err;
    return true;
}

// ------------------------------------------------------------- network ----

struct Buf {
    bf16* p = nullptr;
    int Nb = 0, H = 0, W = 0, C = 0;
    size_t n() const { return static_cast<size_t>(Nb) * H * W * C; }
};

struct ConvLayer {
    std::string name;
    int Co = 0, k = 3, ci_total = 0, nsrc = 1, relu = 1;
    int srcC[2] = {0, 0};      // channels stored per source
    int realC[2] = {0, 0};     // channels with weights (the network input stores in_channels of 8)
    size_t w_off = 0, b_off = 0;
    Buf* in[2] = {nullptr, nullptr};
    Buf* out = nullptr;
    Buf* gin[2] = {nullptr, nullptr};
    Buf* gout = nullptr;
    int out_stride = 0;
    bf16* wf[2] = {nullptr, nullptr};
    int wf_rows = 0;
    int CW[2] = {16, 16}, nch[2] = {0, 0};
    bf16* wd = nullptr;
    int wd_rows = 0, CWz = 16, nchz = 0;
    bool has_dgrad = true;
    bool fwd_dxn = false, bwd_dxn = false;   // column-taps-in-N operands
    ConvPlan fwd, bwd;
    WgradPlan wg;
};

}  // namespace

struct dn_ctx {
    int device = 0, sm_count = 148;
    dn_config cfg{};
    std::string err;
    int L = 4;
    std::vector<std::unique_ptr<Buf>> bufs;
    std::vector<ConvLayer> layers;
    Buf *X = nullptr, *Y = nullptr, *T = nullptr, *dY = nullptr;
    std::vector<Buf*> E0, E1, Pl, U, D0, D1, gE0, gE1, gP, gU, gD0, gD1, gS;
    float *d_params = nullptr, *d_grads = nullptr, *d_m = nullptr, *d_v = nullptr;
    size_t nparams = 0;
    int step = 0;
    double* d_loss = nullptr;
    double* d_partials = nullptr;
    unsigned* d_err = nullptr;
    std::vector<void*> allocs;
};

namespace {

mc_status fail(dn_ctx* c, mc_status s, const std::string& m) {
    if (c) c->err = m;
    return s;
}

#define DN_TRY(ctx, call)                                                                                   \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA,                  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                                \
    } while (0)

template <typename T>
mc_status dalloc(dn_ctx* c, T** p, size_t n) {
    DN_TRY(c, cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T)));
    c->allocs.push_back(*p);
    return MC_OK;
}

mc_status new_buf(dn_ctx* c, Buf** out, int Nb, int H, int W, int C) {
    c->bufs.emplace_back(new Buf());
    Buf* b = c->bufs.back().get();
    b->Nb = Nb; b->H = H; b->W = W; b->C = C;
    mc_status st = dalloc(c, &b->p, b->n());
    if (st != MC_OK) return st;
    DN_TRY(c, cudaMemset(b->p, 0, b->n() * sizeof(bf16)));
    *out = b;
    return MC_OK;
}

// splitmix64 stream -> standard normal by Box-Muller (weight initialisation only)
struct InitRng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (static_cast<double>(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() {
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

mc_status pack_weights(dn_ctx* c, cudaStream_t s) {
    for (ConvLayer& ly : c->layers) {
        const float* w = c->d_params + ly.w_off;
        int coff = 0;
        for (int q = 0; q < ly.nsrc; ++q) {
            if (ly.fwd_dxn)
                DN_TRY(c, dn::launch_pack_dxn(w, ly.Co, ly.ci_total, coff, ly.realC[q], ly.CW[q], ly.nch[q], 0, ly.Co,
                                              ly.wf[q], s));
            else
                DN_TRY(c, dn::launch_pack_fwd(w, ly.Co, ly.wf_rows, ly.k, ly.ci_total, coff, ly.realC[q], ly.CW[q],
                                              ly.nch[q], ly.wf[q], s));
            coff += ly.realC[q];
        }
        if (ly.has_dgrad && ly.bwd_dxn)
            DN_TRY(c, dn::launch_pack_dxn(w, ly.Co, ly.ci_total, 0, ly.Co, ly.CWz, ly.nchz, 1, ly.ci_total, ly.wd, s));
        else if (ly.has_dgrad)
            DN_TRY(c, dn::launch_pack_dgrad(w, ly.Co, ly.k, ly.ci_total, ly.wd_rows, ly.CWz, ly.nchz, ly.wd, s));
    }
    return MC_OK;
}

mc_status run_forward(dn_ctx* c, cudaStream_t s) {
    const int L = c->L;
    size_t li = 0;
    for (int l = 0; l < L; ++l) {
        if (l > 0) {
            const Buf* e = c->E1[l - 1];
            DN_TRY(c, dn::launch_maxpool(e->p, c->Pl[l]->p, e->Nb, e->H, e->W, e->C, s));
        }
        for (int q = 0; q < 2; ++q) {
            ConvLayer& ly = c->layers[li++];
            DN_TRY(c, dn::launch_conv(ly.fwd.ta, ly.fwd.tb, ly.fwd.a, s));
        }
    }
    for (int l = L - 2; l >= 0; --l) {
        const Buf* top = (l == L - 2) ? c->E1[L - 1] : c->D1[l + 1];
        DN_TRY(c, dn::launch_upsample(top->p, c->U[l]->p, top->Nb, top->H, top->W, top->C, s));
        for (int q = 0; q < 2; ++q) {
            ConvLayer& ly = c->layers[li++];
            DN_TRY(c, dn::launch_conv(ly.fwd.ta, ly.fwd.tb, ly.fwd.a, s));
        }
    }
    ConvLayer& out = c->layers[li];
    DN_TRY(c, dn::launch_conv(out.fwd.ta, out.fwd.tb, out.fwd.a, s));
    return MC_OK;
}

mc_status layer_backward(dn_ctx* c, ConvLayer& ly, cudaStream_t s) {
    if (ly.has_dgrad) DN_TRY(c, dn::launch_conv(ly.bwd.ta, ly.bwd.tb, ly.bwd.a, s));
    DN_TRY(c, dn::launch_wgrad(&ly.wg.tz, ly.wg.tx, ly.wg.a, s));
    const Buf* g = ly.gout;
    DN_TRY(c, dn::launch_bias_grad(g->p, g->C, ly.Co, static_cast<long long>(g->Nb) * g->H * g->W,
                                   c->d_grads + ly.b_off, s));
    return MC_OK;
}

mc_status run_backward(dn_ctx* c, cudaStream_t s) {
    const int L = c->L;
    DN_TRY(c, cudaMemsetAsync(c->d_grads, 0, c->nparams * sizeof(float), s));
    const long long npx = static_cast<long long>(c->Y->Nb) * c->Y->H * c->Y->W;
    DN_TRY(c, dn::launch_mse(c->Y->p, c->Y->C, c->T->p, npx, c->dY->p, c->dY->C, c->d_partials, dn::mse_parts(),
                             c->d_loss, s));
    // layer indices: encoder 0..2L-1, decoder levels L-2..0 at 2L + 2(L-2-l), output last
    const int n_layers = static_cast<int>(c->layers.size());
    mc_status st = layer_backward(c, c->layers[n_layers - 1], s);
    if (st != MC_OK) return st;
    for (int l = 0; l <= L - 2; ++l) {
        const int base = 2 * L + 2 * (L - 2 - l);
        st = layer_backward(c, c->layers[base + 1], s);
        if (st != MC_OK) return st;
        st = layer_backward(c, c->layers[base], s);
        if (st != MC_OK) return st;
        Buf* below = (l == L - 2) ? c->gE1[L - 1] : c->gD1[l + 1];
        DN_TRY(c, dn::launch_upsample_bwd(c->gU[l]->p, below->p, below->Nb, below->H, below->W, below->C, s));
    }
    for (int l = L - 1; l >= 0; --l) {
        if (l < L - 1) {
            const Buf* e = c->E1[l];
            DN_TRY(c, dn::launch_maxpool_bwd(e->p, c->gP[l + 1]->p, c->gS[l]->p, c->gE1[l]->p, e->Nb, e->H, e->W,
                                             e->C, s));
        }
        st = layer_backward(c, c->layers[2 * l + 1], s);
        if (st != MC_OK) return st;
        st = layer_backward(c, c->layers[2 * l], s);
        if (st != MC_OK) return st;
    }
    return MC_OK;
}

mc_status check_err(dn_ctx* c) {
    unsigned e = 0;
    DN_TRY(c, cudaMemcpy(&e, c->d_err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e) return fail(c, MC_ERR_TIMEOUT, "a bounded tensor-core pipeline wait gave up (code " + std::to_string(e) + ")");
    return MC_OK;
}

mc_status build(dn_ctx* c) {
    const dn_config& g = c->cfg;
    const int L = g.levels, Nb = g.batch;
    c->L = L;
    const int H0 = g.height, W0 = g.width;
    auto ch = [&](int l) { return g.base_channels << l; };
    auto hl = [&](int l) { return H0 >> l; };
    auto wl = [&](int l) { return W0 >> l; };
    c->E0.assign(L, nullptr); c->E1.assign(L, nullptr); c->Pl.assign(L, nullptr); c->U.assign(L, nullptr);
    c->D0.assign(L, nullptr); c->D1.assign(L, nullptr); c->gE0.assign(L, nullptr); c->gE1.assign(L, nullptr);
    c->gP.assign(L, nullptr); c->gU.assign(L, nullptr); c->gD0.assign(L, nullptr); c->gD1.assign(L, nullptr);
    c->gS.assign(L, nullptr);
    mc_status st;
#define NB(ptr, h, w, cc)                                  \
    do {                                                   \
        st = new_buf(c, &(ptr), Nb, (h), (w), (cc));       \
        if (st != MC_OK) return st;                        \
    } while (0)
    NB(c->X, H0, W0, 8);
    NB(c->Y, H0, W0, 1);
    NB(c->T, H0, W0, 1);
    NB(c->dY, H0, W0, 8);
    for (int l = 0; l < L; ++l) {
        NB(c->E0[l], hl(l), wl(l), ch(l));
        NB(c->E1[l], hl(l), wl(l), ch(l));
        NB(c->gE0[l], hl(l), wl(l), ch(l));
        NB(c->gE1[l], hl(l), wl(l), ch(l));
        if (l > 0) {
            NB(c->Pl[l], hl(l), wl(l), ch(l - 1));
            NB(c->gP[l], hl(l), wl(l), ch(l - 1));
        }
        if (l < L - 1) {
            NB(c->U[l], hl(l), wl(l), ch(l + 1));
            NB(c->gU[l], hl(l), wl(l), ch(l + 1));
            NB(c->D0[l], hl(l), wl(l), ch(l));
            NB(c->D1[l], hl(l), wl(l), ch(l));
            NB(c->gD0[l], hl(l), wl(l), ch(l));
            NB(c->gD1[l], hl(l), wl(l), ch(l));
            NB(c->gS[l], hl(l), wl(l), ch(l));
        }
    }
#undef NB
    // layers in parameter order
    auto add = [&](const char* name, int Co, int k, int nsrc, Buf* in0, Buf* in1, Buf* out, Buf* gin0, Buf* gin1,
                   Buf* gout, int relu) {
        ConvLayer ly;
        ly.name = name;
        ly.Co = Co; ly.k = k; ly.nsrc = nsrc; ly.relu = relu;
        ly.in[0] = in0; ly.in[1] = in1; ly.out = out; ly.gin[0] = gin0; ly.gin[1] = gin1; ly.gout = gout;
        ly.srcC[0] = in0->C;
        ly.srcC[1] = in1 ? in1->C : 0;
        c->layers.push_back(ly);
    };
    char nm[32];
    for (int l = 0; l < L; ++l) {
        Buf* in = (l == 0) ? c->X : c->Pl[l];
        snprintf(nm, sizeof(nm), "enc%da", l);
        add(nm, ch(l), 3, 1, in, nullptr, c->E0[l], l == 0 ? nullptr : c->gP[l], nullptr, c->gE0[l], 1);
        snprintf(nm, sizeof(nm), "enc%db", l);
        add(nm, ch(l), 3, 1, c->E0[l], nullptr, c->E1[l], c->gE0[l], nullptr, c->gE1[l], 1);
    }
    for (int l = L - 2; l >= 0; --l) {
        snprintf(nm, sizeof(nm), "dec%da", l);
        add(nm, ch(l), 3, 2, c->U[l], c->E1[l], c->D0[l], c->gU[l], c->gS[l], c->gD0[l], 1);
        snprintf(nm, sizeof(nm), "dec%db", l);
        add(nm, ch(l), 3, 1, c->D0[l], nullptr, c->D1[l], c->gD0[l], nullptr, c->gD1[l], 1);
    }
    add("out", 1, 1, 1, c->D1[0], nullptr, c->Y, c->gD1[0], nullptr, c->dY, 0);

    // parameter offsets (weights [Co][k][k][Ci] then biases); the network input
    // has in_channels real channels of the 8 stored
    size_t off = 0;
    for (ConvLayer& ly : c->layers) {
        for (int q = 0; q < ly.nsrc; ++q) ly.realC[q] = (ly.in[q] == c->X) ? c->cfg.in_channels : ly.srcC[q];
        ly.ci_total = ly.realC[0] + ly.realC[1];
        ly.w_off = off;
        off += static_cast<size_t>(ly.Co) * ly.k * ly.k * ly.ci_total;
        ly.b_off = off;
        off += ly.Co;
    }
    c->nparams = off;
    if ((st = dalloc(c, &c->d_params, off)) != MC_OK) return st;
    if ((st = dalloc(c, &c->d_grads, off)) != MC_OK) return st;
    if ((st = dalloc(c, &c->d_m, off)) != MC_OK) return st;
    if ((st = dalloc(c, &c->d_v, off)) != MC_OK) return st;
    if ((st = dalloc(c, &c->d_loss, 1)) != MC_OK) return st;
    if ((st = dalloc(c, &c->d_partials, dn::mse_parts())) != MC_OK) return st;
    if ((st = dalloc(c, &c->d_err, 1)) != MC_OK) return st;
    DN_TRY(c, cudaMemset(c->d_err, 0, sizeof(unsigned)));
    DN_TRY(c, cudaMemset(c->d_m, 0, off * sizeof(float)));
    DN_TRY(c, cudaMemset(c->d_v, 0, off * sizeof(float)));

    // packed operands and launch plans
    for (ConvLayer& ly : c->layers) {
        int nt_f, tiles_f;
        n_tiling(ly.Co, nt_f, tiles_f);
        ly.wf_rows = nt_f * tiles_f;
        ly.fwd_dxn = dxn_fits(ly.k, ly.Co, ly.nsrc, ly.srcC);
        for (int q = 0; q < ly.nsrc; ++q) {
            // the network input's 8 stored channels hold 1 real one: its weight
            // operand has zeros for the other 7
            ly.CW[q] = cw_for(ly.srcC[q]);
            ly.nch[q] = chunks(ly.srcC[q], ly.CW[q]);
            const size_t n_op = ly.fwd_dxn ? static_cast<size_t>(3 * ly.Co) * 3 * ly.nch[q] * ly.CW[q]
                                           : static_cast<size_t>(ly.wf_rows) * ly.k * ly.k * ly.nch[q] * ly.CW[q];
            if ((st = dalloc(c, &ly.wf[q], n_op)) != MC_OK) return st;
        }
        ly.has_dgrad = ly.gin[0] != nullptr;
        const int Cz = ly.gout->C;
        ly.CWz = cw_for(Cz);
        ly.nchz = chunks(Cz, ly.CWz);
        int nt_d, tiles_d;
        n_tiling(ly.srcC[0] + ly.srcC[1], nt_d, tiles_d);
        ly.wd_rows = nt_d * tiles_d;
        const int zC1[2] = {Cz, 0};
        ly.bwd_dxn = ly.has_dgrad && dxn_fits(ly.k, ly.srcC[0] + ly.srcC[1], 1, zC1);
        const size_t n_wd = ly.bwd_dxn ? static_cast<size_t>(3 * (ly.srcC[0] + ly.srcC[1])) * 3 * ly.nchz * ly.CWz
                                       : static_cast<size_t>(ly.wd_rows) * ly.k * ly.k * ly.nchz * ly.CWz;
        if (ly.has_dgrad && (st = dalloc(c, &ly.wd, n_wd)) != MC_OK) return st;
        const Buf* o = ly.out;
        const bf16* srcs[2] = {ly.in[0]->p, ly.in[1] ? ly.in[1]->p : nullptr};
        const bf16* wops[2] = {ly.wf[0], ly.wf[1]};
        bf16* dsts[2] = {o->p, nullptr};
        const int dC[2] = {o->C, 0};
        if (!plan_conv(ly.fwd, ly.nsrc, srcs, ly.srcC, o->Nb, o->H, o->W, ly.k, wops, ly.wf_rows, ly.Co,
                       c->d_params + ly.b_off, ly.relu, 1, ly.Co, dsts, dC, nullptr, c->d_err, c->sm_count, true,
                       ly.fwd_dxn))
            return fail(c, MC_ERR_CUDA, "tensor map encoding failed (" + ly.name + ")");
        if (ly.has_dgrad) {
            const bf16* zs[2] = {ly.gout->p, nullptr};
            const bf16* wd2[2] = {ly.wd, nullptr};
            const int zC[2] = {Cz, 0};
            bf16* gd[2] = {ly.gin[0]->p, ly.gin[1] ? ly.gin[1]->p : nullptr};
            const int gC[2] = {ly.srcC[0], ly.srcC[1]};
            const bf16* mk[2] = {ly.in[0]->p, ly.in[1] ? ly.in[1]->p : nullptr};
            if (!plan_conv(ly.bwd, 1, zs, zC, o->Nb, o->H, o->W, ly.k, wd2, ly.wd_rows, ly.srcC[0] + ly.srcC[1],
                           nullptr, 0, ly.nsrc, ly.srcC[0], gd, gC, mk, c->d_err, c->sm_count, true, ly.bwd_dxn))
                return fail(c, MC_ERR_CUDA, "tensor map encoding failed (" + ly.name + " dgrad)");
        }
        if (!plan_wgrad(ly.wg, ly.gout->p, Cz, ly.Co, ly.nsrc, srcs, ly.srcC, o->Nb, o->H, o->W, ly.k,
                        c->d_grads + ly.w_off, c->d_err, c->sm_count))
            return fail(c, MC_ERR_CUDA, "tensor map encoding failed (" + ly.name + " wgrad)");
        // the network input's gradient operand spans the 8 stored channels but
        // only the first in_channels have weights: restrict the weight gradient to them
        if (ly.in[0] == c->X) {
            ly.wg.a.src_C[0] = c->cfg.in_channels;
            ly.wg.a.ci_total = c->cfg.in_channels;
        }
    }
    return MC_OK;
}

mc_status init_params(dn_ctx* c) {
    std::vector<float> h(c->nparams, 0.0f);
    InitRng r{c->cfg.seed * 0x9E3779B97F4A7C15ull + 1};
    for (const ConvLayer& ly : c->layers) {
        const double fan_in = static_cast<double>(ly.k) * ly.k * ly.ci_total;
        const double sd = std::sqrt((ly.relu ? 2.0 : 1.0) / fan_in);
        const size_t nw = static_cast<size_t>(ly.Co) * ly.k * ly.k * ly.ci_total;
        for (size_t i = 0; i < nw; ++i) h[ly.w_off + i] = static_cast<float>(sd * r.normal());
    }
    DN_TRY(c, cudaMemcpy(c->d_params, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    return pack_weights(c, nullptr);
}

}  // namespace

extern "C" {

void dn_config_default(dn_config* cfg) {
    if (!cfg) return;
    cfg->height = 768;
    cfg->width = 1024;
    cfg->batch = 1;
    cfg->levels = 4;
    cfg->base_channels = 32;
    cfg->in_channels = 1;
    cfg->seed = 1;
}

const char* dn_last_error(const dn_ctx* c) { return c ? c->err.c_str() : "null context"; }

mc_status dn_create(const dn_config* cfg_in, int device, dn_ctx** out) {
    if (!out) return MC_ERR_ARG;
    *out = nullptr;
    dn_config cfg;
    if (cfg_in) cfg = *cfg_in; else dn_config_default(&cfg);
    if (cfg.levels < 2 || cfg.levels > 5 || cfg.batch < 1 || cfg.base_channels < 32 || cfg.base_channels % 32 != 0 ||
        (cfg.base_channels << (cfg.levels - 1)) > 256 || cfg.in_channels < 1 || cfg.in_channels > 8)
        return MC_ERR_ARG;
    const int m = 1 << (cfg.levels - 1);
    if (cfg.height < m || cfg.width < m || cfg.height % m != 0 || cfg.width % m != 0 || cfg.height > 16384 ||
        cfg.width > 16384)
        return MC_ERR_ARG;
    dn_ctx* c = new dn_ctx();
    c->cfg = cfg;
    c->device = device;
    auto bail = [&](mc_status s) {
        dn_destroy(c);
        return s;
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(MC_ERR_CUDA);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (!encoder()) return bail(MC_ERR_CUDA);
    if (dn::conv_prepare() != cudaSuccess) return bail(MC_ERR_CUDA);
    mc_status st = build(c);
    if (st == MC_OK) st = init_params(c);
    if (st == MC_OK && cudaDeviceSynchronize() != cudaSuccess) st = MC_ERR_CUDA;
    if (st != MC_OK) return bail(st);
    *out = c;
    return MC_OK;
}

mc_status dn_destroy(dn_ctx* c) {
    if (!c) return MC_OK;
    cudaSetDevice(c->device);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
    return MC_OK;
}

mc_status dn_param_count(const dn_ctx* c, size_t* n) {
    if (!c || !n) return MC_ERR_ARG;
    *n = c->nparams;
    return MC_OK;
}

mc_status dn_set_params(dn_ctx* c, const float* p, size_t n) {
    if (!c) return MC_ERR_ARG;
    if (!p || n != c->nparams) return fail(c, MC_ERR_ARG, "parameter count mismatch");
    DN_TRY(c, cudaSetDevice(c->device));
    DN_TRY(c, cudaMemcpy(c->d_params, p, n * sizeof(float), cudaMemcpyHostToDevice));
    DN_TRY(c, cudaMemset(c->d_m, 0, n * sizeof(float)));
    DN_TRY(c, cudaMemset(c->d_v, 0, n * sizeof(float)));
    c->step = 0;
    mc_status st = pack_weights(c, nullptr);
    if (st != MC_OK) return st;
    DN_TRY(c, cudaDeviceSynchronize());
    return MC_OK;
}

mc_status dn_get_params(dn_ctx* c, float* p, size_t n) {
    if (!c) return MC_ERR_ARG;
    if (!p || n != c->nparams) return fail(c, MC_ERR_ARG, "parameter count mismatch");
    DN_TRY(c, cudaSetDevice(c->device));
    DN_TRY(c, cudaMemcpy(p, c->d_params, n * sizeof(float), cudaMemcpyDeviceToHost));
    return MC_OK;
}

mc_status dn_get_grads(dn_ctx* c, float* g, size_t n) {
    if (!c) return MC_ERR_ARG;
    if (!g || n != c->nparams) return fail(c, MC_ERR_ARG, "parameter count mismatch");
    DN_TRY(c, cudaSetDevice(c->device));
    DN_TRY(c, cudaMemcpy(g, c->d_grads, n * sizeof(float), cudaMemcpyDeviceToHost));
    return check_err(c);
}

mc_status dn_forward(dn_ctx* c, const float* input, float in_scale, float* output, float out_scale, void* stream) {
    if (!c) return MC_ERR_ARG;
    if (!input || !output) return fail(c, MC_ERR_ARG, "null pointer");
    DN_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long hw = static_cast<long long>(c->X->H) * c->X->W, npx = c->X->Nb * hw;
    DN_TRY(c, dn::launch_prep(input, c->cfg.in_channels, hw, in_scale, npx, c->X->p, c->X->C, s));
    mc_status st = run_forward(c, s);
    if (st != MC_OK) return st;
    DN_TRY(c, dn::launch_to_f32(c->Y->p, c->Y->C, npx, out_scale, output, s));
    return MC_OK;
}

mc_status dn_get_output(dn_ctx* c, float* out, void* stream) {
    if (!c || !out) return MC_ERR_ARG;
    DN_TRY(c, cudaSetDevice(c->device));
    const long long npx = static_cast<long long>(c->Y->Nb) * c->Y->H * c->Y->W;
    DN_TRY(c, dn::launch_to_f32(c->Y->p, c->Y->C, npx, 1.0f, out, static_cast<cudaStream_t>(stream)));
    return MC_OK;
}

mc_status dn_train_step(dn_ctx* c, const float* input, const float* target, float in_scale, float lr, double* loss,
                        void* stream) {
    if (!c) return MC_ERR_ARG;
    if (!input || !target) return fail(c, MC_ERR_ARG, "null pointer");
    if (!(lr >= 0.0f)) return fail(c, MC_ERR_ARG, "learning rate must be >= 0");
    DN_TRY(c, cudaSetDevice(c->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long hw = static_cast<long long>(c->X->H) * c->X->W, npx = c->X->Nb * hw;
    DN_TRY(c, dn::launch_prep(input, c->cfg.in_channels, hw, in_scale, npx, c->X->p, c->X->C, s));
    DN_TRY(c, dn::launch_prep(target, 1, hw, in_scale, npx, c->T->p, 1, s));
    mc_status st = run_forward(c, s);
    if (st != MC_OK) return st;
    st = run_backward(c, s);
    if (st != MC_OK) return st;
    ++c->step;
    const double c1 = 1.0 - std::pow(0.9, c->step), c2 = 1.0 - std::pow(0.999, c->step);
    DN_TRY(c, dn::launch_adam(c->d_params, c->d_grads, c->d_m, c->d_v, static_cast<long long>(c->nparams), lr, 0.9f,
                              0.999f, 1e-8f, static_cast<float>(c1), static_cast<float>(c2), s));
    st = pack_weights(c, s);
    if (st != MC_OK) return st;
    if (loss) {
        DN_TRY(c, cudaMemcpyAsync(loss, c->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        DN_TRY(c, cudaStreamSynchronize(s));
        return check_err(c);
    }
    return MC_OK;
}

}  // extern "C"

// ---------------------------------------------------------- primitives ----

namespace {

struct Scratch {
    std::vector<void*> p;
    ~Scratch() {
        for (void* q : p) cudaFree(q);
    }
    template <typename T>
    T* get(size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        p.push_back(q);
        return static_cast<T*>(q);
    }
};

mc_status prim_check(cudaStream_t s, unsigned* err) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return MC_ERR_CUDA;
    unsigned e = 0;
    if (cudaMemcpy(&e, err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) return MC_ERR_CUDA;
    return e ? MC_ERR_TIMEOUT : MC_OK;
}

bool chan_ok(int c) { return c > 0 && c % 8 == 0 && (c < 64 || c % 64 == 0) && c <= 1024; }

int device_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

extern "C" {


mc_status dn_conv2d_forward(const uint16_t* x0, int c0, const uint16_t* x1, int c1, int batch, int height,
                            int width, const float* weight, const float* bias, int k, int co, int relu, uint16_t* y,
                            int y_stride, void* stream) {
    if (!x0 || !weight || !y || !chan_ok(c0) || (x1 && !chan_ok(c1)) || (k != 1 && k != 3) || co < 1 ||
        co > 1024 || y_stride < co || batch < 1 || height < 1 || width < 1)
        return MC_ERR_ARG;
    if (!encoder() || dn::conv_prepare() != cudaSuccess) return MC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    const int nsrc = x1 ? 2 : 1;
    const int C[2] = {c0, x1 ? c1 : 0};
    int nt, tiles;
    n_tiling(co, nt, tiles);
    const int rows = nt * tiles;
    bf16* wop[2] = {nullptr, nullptr};
    unsigned* err = sc.get<unsigned>(1);
    if (!err || cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) return MC_ERR_CUDA;
    int coff = 0;
    const bool dxn = dxn_fits(k, co, nsrc, C);
    for (int q = 0; q < nsrc; ++q) {
        const int CW = cw_for(C[q]), nch = chunks(C[q], CW);
        wop[q] = sc.get<bf16>(dxn ? static_cast<size_t>(3 * co) * 3 * nch * CW
                                  : static_cast<size_t>(rows) * k * k * nch * CW);
        if (!wop[q]) return MC_ERR_OOM;
        const cudaError_t e = dxn ? dn::launch_pack_dxn(weight, co, C[0] + C[1], coff, C[q], CW, nch, 0, co, wop[q], s)
                                  : dn::launch_pack_fwd(weight, co, rows, k, C[0] + C[1], coff, C[q], CW, nch, wop[q], s);
        if (e != cudaSuccess) return MC_ERR_CUDA;
        coff += C[q];
    }
    ConvPlan P;
    const bf16* srcs[2] = {reinterpret_cast<const bf16*>(x0), reinterpret_cast<const bf16*>(x1)};
    const bf16* wops[2] = {wop[0], wop[1]};
    bf16* dst[2] = {reinterpret_cast<bf16*>(y), nullptr};
    const int dC[2] = {y_stride, 0};
    if (!plan_conv(P, nsrc, srcs, C, batch, height, width, k, wops, rows, co, bias, relu, 1, co, dst, dC, nullptr,
                   err, device_sms(), true, dxn))
        return MC_ERR_CUDA;
    if (dn::launch_conv(P.ta, P.tb, P.a, s) != cudaSuccess) return MC_ERR_CUDA;
    return prim_check(s, err);
}

mc_status dn_conv2d_backward_data(const uint16_t* dz, int dz_stride, int co, int batch, int height, int width,
                                  const float* weight, int k, uint16_t* dx0, int c0, const uint16_t* mask0,
                                  uint16_t* dx1, int c1, const uint16_t* mask1, void* stream) {
    if (!dz || !weight || !dx0 || !chan_ok(c0) || (dx1 && !chan_ok(c1)) || (k != 1 && k != 3) || co < 1 ||
        dz_stride < co || dz_stride % 8 != 0 || batch < 1 || height < 1 || width < 1)
        return MC_ERR_ARG;
    if (!encoder() || dn::conv_prepare() != cudaSuccess) return MC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    const int ndst = dx1 ? 2 : 1;
    const int ci_total = c0 + (dx1 ? c1 : 0);
    const int CWz = cw_for(dz_stride), nchz = chunks(dz_stride, CWz);
    int nt, tiles;
    n_tiling(ci_total, nt, tiles);
    const int rows = nt * tiles;
    const int zC1[2] = {dz_stride, 0};
    const bool dxn = dxn_fits(k, ci_total, 1, zC1);
    unsigned* err = sc.get<unsigned>(1);
    bf16* wd = sc.get<bf16>(dxn ? static_cast<size_t>(3 * ci_total) * 3 * nchz * CWz
                                : static_cast<size_t>(rows) * k * k * nchz * CWz);
    if (!err || !wd) return MC_ERR_OOM;
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) return MC_ERR_CUDA;
    const cudaError_t pe = dxn ? dn::launch_pack_dxn(weight, co, ci_total, 0, co, CWz, nchz, 1, ci_total, wd, s)
                               : dn::launch_pack_dgrad(weight, co, k, ci_total, rows, CWz, nchz, wd, s);
    if (pe != cudaSuccess) return MC_ERR_CUDA;
    ConvPlan P;
    const bf16* zs[2] = {reinterpret_cast<const bf16*>(dz), nullptr};
    const bf16* w2[2] = {wd, nullptr};
    const int zC[2] = {dz_stride, 0};
    bf16* dst[2] = {reinterpret_cast<bf16*>(dx0), reinterpret_cast<bf16*>(dx1)};
    const int dC[2] = {c0, dx1 ? c1 : 0};
    const bf16* mk[2] = {reinterpret_cast<const bf16*>(mask0), reinterpret_cast<const bf16*>(mask1)};
    if (!plan_conv(P, 1, zs, zC, batch, height, width, k, w2, rows, ci_total, nullptr, 0, ndst, c0, dst, dC, mk, err,
                   device_sms(), true, dxn))
        return MC_ERR_CUDA;
    if (dn::launch_conv(P.ta, P.tb, P.a, s) != cudaSuccess) return MC_ERR_CUDA;
    return prim_check(s, err);
}

mc_status dn_conv2d_backward_weights(const uint16_t* dz, int dz_stride, int co, const uint16_t* x0, int c0,
                                     const uint16_t* x1, int c1, int batch, int height, int width, int k, float* dw,
                                     float* db, void* stream) {
    if (!dz || !x0 || !dw || !chan_ok(c0) || (x1 && !chan_ok(c1)) || (k != 1 && k != 3) || co < 1 ||
        dz_stride < co || dz_stride % 8 != 0 || batch < 1 || height < 1 || width < 1)
        return MC_ERR_ARG;
    if (db && !(co == 1 || co == 32 || co == 64 || co == 128 || co == 256)) return MC_ERR_ARG;
    if (!encoder() || dn::conv_prepare() != cudaSuccess) return MC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    unsigned* err = sc.get<unsigned>(1);
    if (!err || cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) return MC_ERR_CUDA;
    int sms = 148;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    WgradPlan P;
    const int nsrc = x1 ? 2 : 1;
    const bf16* srcs[2] = {reinterpret_cast<const bf16*>(x0), reinterpret_cast<const bf16*>(x1)};
    const int C[2] = {c0, x1 ? c1 : 0};
    if (!plan_wgrad(P, reinterpret_cast<const bf16*>(dz), dz_stride, co, nsrc, srcs, C, batch, height, width, k, dw,
                    err, sms))
        return MC_ERR_CUDA;
    if (dn::launch_wgrad(&P.tz, P.tx, P.a, s) != cudaSuccess) return MC_ERR_CUDA;
    if (db && dn::launch_bias_grad(reinterpret_cast<const bf16*>(dz), dz_stride, co,
                                   static_cast<long long>(batch) * height * width, db, s) != cudaSuccess)
        return MC_ERR_CUDA;
    return prim_check(s, err);
}

mc_status dn_maxpool2(const uint16_t* x, uint16_t* y, int batch, int height, int width, int c, void* stream) {
    if (!x || !y || c % 8 || c < 8 || height % 2 || width % 2 || batch < 1 || height < 2 || width < 2)
        return MC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dn::launch_maxpool(reinterpret_cast<const bf16*>(x), reinterpret_cast<bf16*>(y), batch, height, width, c,
                           s) != cudaSuccess)
        return MC_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

mc_status dn_maxpool2_backward(const uint16_t* x, const uint16_t* dy, const uint16_t* add, uint16_t* dx, int batch,
                               int height, int width, int c, void* stream) {
    if (!x || !dy || !dx || c % 8 || c < 8 || height % 2 || width % 2 || batch < 1 || height < 2 || width < 2)
        return MC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dn::launch_maxpool_bwd(reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(dy),
                               reinterpret_cast<const bf16*>(add), reinterpret_cast<bf16*>(dx), batch, height, width,
                               c, s) != cudaSuccess)
        return MC_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

mc_status dn_upsample2(const uint16_t* x, uint16_t* y, int batch, int height, int width, int c, void* stream) {
    if (!x || !y || c % 8 || c < 8 || batch < 1 || height < 1 || width < 1) return MC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dn::launch_upsample(reinterpret_cast<const bf16*>(x), reinterpret_cast<bf16*>(y), batch, height, width, c,
                            s) != cudaSuccess)
        return MC_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

mc_status dn_upsample2_backward(const uint16_t* dy, uint16_t* dx, int batch, int height, int width, int c,
                                void* stream) {
    if (!dy || !dx || c % 8 || c < 8 || batch < 1 || height < 1 || width < 1) return MC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dn::launch_upsample_bwd(reinterpret_cast<const bf16*>(dy), reinterpret_cast<bf16*>(dx), batch, height,
                                width, c, s) != cudaSuccess)
        return MC_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

}  // extern "C"
