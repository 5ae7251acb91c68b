// Kernels of the EPID-image denoiser (a 2D U-Net trained on pairs of
// low- and high-count Monte Carlo images).
//
// Convolutions run on the fifth-generation tensor cores as implicit GEMMs:
//   forward / input gradient: M = 128 pixels of one image row (a TMA box of
//     the NHWC activation shifted by the tap offset; zero fill supplies the
//     padding), N = output channels, K = taps x input channels.  A producer
//     thread streams (activation, weight) tile pairs through a ring of
//     shared-memory stages with TMA; one thread per column slice issues
//     tcgen05.mma into a TMEM accumulator; four warps read the accumulator
//     back (tcgen05.ld) and apply
//     the epilogue (bias, ReLU, the ReLU mask of the layer below, the split of
//     a concatenated input, bf16 rounding).
//   weight gradient: M = 128 output channels, N = 64 input channels, K =
//     pixels; both operands are read channel-contiguous (MN-major) straight
//     from the NHWC tensors, one tap row per CTA with its three column taps
//     in three TMEM accumulators, split over pixel ranges and reduced with
//     f32 atomics.
// Everything else (pooling, upsampling, loss, Adam, weight packing) is
// HBM-bound pointwise work on CUDA cores.
#include "dn_kernels.cuh"

#include <algorithm>
#include "dn_tc.cuh"

namespace dn {

namespace {

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    const uint32_t a = smem_u32(p);
    return p + ((1024u - (a & 1023u)) & 1023u);
}

// The mask words the vector path of epilogue16 reads for columns co0 ..
// co0+15 of one pixel, loaded ahead so their latency overlaps the TMEM read.
__device__ __forceinline__ void epi_mask16(const ConvArgs& a, int co0, size_t pix, uint4* mv) {
    const int d = (a.ndst > 1 && co0 >= a.dst_split) ? 1 : 0;
    const int cc0 = co0 - (d ? a.dst_split : 0);
    const int dC = a.dst_C[d];
    const int dend = d ? a.N : (a.ndst > 1 ? a.dst_split : a.N);
    const __nv_bfloat16* mk = a.mask[d];
    if (mk && co0 + 16 <= dend && (dC & 7) == 0 && (cc0 & 7) == 0) {
        const uint4* m = reinterpret_cast<const uint4*>(mk + pix * dC + cc0);
        mv[0] = __ldg(m);
        mv[1] = __ldg(m + 1);
    }
}

// Epilogue of 16 accumulator columns (output channels co0 .. co0+15) of one
// pixel: bias, ReLU, the mask of the source layer, the split of a
// concatenated input, bf16 rounding; 16-byte stores where aligned.  mvp: the
// mask words from epi_mask16, or null to load them here.
__device__ __forceinline__ void epilogue16(const ConvArgs& a, const float* bias, const float* v, int co0, size_t pix,
                                           const uint4* mvp = nullptr) {
    const int d = (a.ndst > 1 && co0 >= a.dst_split) ? 1 : 0;
    const int cc0 = co0 - (d ? a.dst_split : 0);
    const int dC = a.dst_C[d];
    const int dend = d ? a.N : (a.ndst > 1 ? a.dst_split : a.N);
    __nv_bfloat16* out = a.dst[d] + pix * dC;
    const __nv_bfloat16* mk = a.mask[d] ? a.mask[d] + pix * dC : nullptr;
    if (co0 + 16 <= dend && (dC & 7) == 0 && (cc0 & 7) == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint4 mv = make_uint4(0, 0, 0, 0);
            if (mk) mv = mvp ? mvp[h] : *reinterpret_cast<const uint4*>(mk + cc0 + 8 * h);
            const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mv);
            __align__(16) __nv_bfloat16 o[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float val = v[8 * h + j];
                if (a.bias) val += bias[co0 + 8 * h + j];
                if (a.relu) val = fmaxf(val, 0.0f);
                if (mk && !(__bfloat162float(mb[j]) > 0.0f)) val = 0.0f;
                o[j] = __float2bfloat16_rn(val);
            }
            *reinterpret_cast<uint4*>(out + cc0 + 8 * h) = *reinterpret_cast<const uint4*>(o);
        }
    } else {
        for (int j = 0; j < 16; ++j) {
            const int co = co0 + j;
            if (co >= a.N) break;
            const int dd = (a.ndst > 1 && co >= a.dst_split) ? 1 : 0;
            const int cc = co - (dd ? a.dst_split : 0);
            float val = v[j];
            if (a.bias) val += bias[co];
            if (a.relu) val = fmaxf(val, 0.0f);
            const size_t o = pix * a.dst_C[dd] + cc;
            if (a.mask[dd] && !(__bfloat162float(a.mask[dd][o]) > 0.0f)) val = 0.0f;
            a.dst[dd][o] = __float2bfloat16_rn(val);
        }
    }
}

}  // namespace

// ------------------------------------------------------- convolution ------

// Persistent: CTA b takes output tiles b, b + grid, ...; a tile is 128
// pixels of one image row x N_tile output channels.  Warp 0 (one lane)
// streams the (activation, weight) tile pairs of every K step of every tile
// through a ring of `stages` shared-memory slots; warps 1 .. n_issue (one lane
// each) issue the MMAs of a tile, one column slice each, into one of two TMEM
// accumulators; warps 4-7 and 8-11 drain the accumulators (tcgen05.ld), so a
// tile's epilogue overlaps the next tile's MMAs.
__global__ void __launch_bounds__(kConvMaxThreads) k_conv(const __grid_constant__ CUtensorMap ta0,
                                              const __grid_constant__ CUtensorMap ta1,
                                              const __grid_constant__ CUtensorMap tb0,
                                              const __grid_constant__ CUtensorMap tb1, const ConvArgs a) {
    extern __shared__ uint8_t dsm[];
    uint8_t* tiles = align1024(dsm);
    const int S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(tiles + S * a.stage_bytes);
    uint64_t* empty = full + S;
    const int GE = a.epi_groups;     // accumulator buffers = epilogue warpgroups
    uint64_t* accf = empty + S;      // [GE] accumulator ready (MMA -> epilogue)
    uint64_t* acce = accf + GE;      // [GE] accumulator drained (epilogue -> MMA)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + GE);
    volatile uint32_t* abort_flag = tslot + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ float s_bias[kConvMaxN];                  // the epilogue's bias, read once
    if (a.bias)
        for (int i = threadIdx.x; i < a.N; i += blockDim.x) s_bias[i] = __ldg(&a.bias[i]);

    const int segs = (a.W + 127) >> 7;
    const int n_tiles = (a.N + a.N_tile - 1) / a.N_tile;
    const int total = segs * a.H * a.Nb * n_tiles;
    const int p = a.k >> 1;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], a.n_issue);
        }
        for (int i = 0; i < GE; ++i) {
            mbar_init(&accf[i], a.n_issue);
            mbar_init(&acce[i], 4);
        }
        *abort_flag = 0u;
        mbar_fence_init();
        tma_prefetch(&ta0);
        tma_prefetch(&tb0);
        if (a.nsrc > 1) {
            tma_prefetch(&ta1);
            tma_prefetch(&tb1);
        }
    }
    if (warp == 1) tmem_alloc(tslot, static_cast<uint32_t>(a.tmem_cols));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // tile t -> (x segment, row, image, N tile); N tiles outermost so that
    // neighbouring CTAs share input rows in L2
    auto decode = [&](int t, int& x0, int& y, int& n, int& n0) {
        const int per = segs * a.H * a.Nb;
        const int nt = t / per;
        int r = t - nt * per;
        const int xs = r % segs;
        r /= segs;
        y = r % a.H;
        n = r / a.H;
        x0 = xs << 7;
        n0 = nt * a.N_tile;
    };

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0, st = 0, ph = 0;
            const int nch0 = a.src[0].nch, chunks = nch0 + (a.nsrc > 1 ? a.src[1].nch : 0);
            for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
                int x0, y, n, n0;
                decode(t, x0, y, n, n0);
                int tap = 0, dy = 0, dx = 0, r = 0;          // K step i = (tap, chunk r), counted
                for (int i = 0; i < a.nk; ++i, ++it) {
                    if (it >= static_cast<uint32_t>(S) && !mbar_wait(&empty[st], ph ^ 1u, a.err, kErrWaitEmpty)) {
                        *abort_flag = 1u;
                        break;
                    }
                    const int s_ = r < nch0 ? 0 : 1, ch = s_ ? r - nch0 : r;
                    const ConvSrc& src = a.src[s_];
                    uint8_t* sa = tiles + st * a.stage_bytes;
                    uint8_t* sb = sa + a.a_region;
                    const uint32_t bytes =
                        (128u + static_cast<uint32_t>(a.N_tile)) * static_cast<uint32_t>(src.CW) * 2u;
                    mbar_expect_tx(&full[st], bytes);
                    tma_load_4d(sa, s_ ? &ta1 : &ta0, &full[st], ch * src.CW, x0 + dx - p, y + dy - p, n);
                    tma_load_2d(sb, s_ ? &tb1 : &tb0, &full[st], (tap * src.nch + ch) * src.CW, n0);
                    if (++st == static_cast<uint32_t>(S)) { st = 0; ph ^= 1u; }
                    if (++r == chunks) { r = 0; ++tap; if (++dx == a.k) { dx = 0; ++dy; } }
                }
                if (*abort_flag) break;
            }
            // every copy this CTA started has landed before it may exit
            const uint32_t issued = it;
            for (uint32_t st = 0; st < static_cast<uint32_t>(S) && st < issued; ++st) {
                const uint32_t last = st + ((issued - 1 - st) / S) * S;
                mbar_wait(&full[st], (last / S) & 1, a.err, kErrWaitTail);
            }
        }
    } else if (warp <= 3) {
        // MMA warps 1 .. n_issue: warp 1 + js issues column slice js of every
        // tile.  The descriptors of stage 0 are built once per source; a stage
        // adds its offset and each 16-channel slice 32 bytes (2 descriptor
        // units), so the issuing thread's loop stays short.
        const uint32_t js = static_cast<uint32_t>(warp - 1);
        if (lane == 0 && warp <= a.n_issue) {
            const uint32_t t0 = smem_u32(tiles);
            uint64_t da_s[2], db_s[2];
            int n16_s[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int CW = a.src[q < a.nsrc ? q : 0].CW;
                const uint32_t row = static_cast<uint32_t>(CW) * 2u, swz = swz_for_row(row);
                da_s[q] = smem_desc(t0, 16u, 8u * row, swz);
                db_s[q] = smem_desc(t0 + a.a_region + js * static_cast<uint32_t>(a.n_slice) * row, 16u, 8u * row, swz);
                n16_s[q] = CW / 16;
            }
            const uint64_t stage_units = a.stage_bytes >> 4;
            const int nch0 = a.src[0].nch, chunks = nch0 + (a.nsrc > 1 ? a.src[1].nch : 0);
            uint32_t st = 0, ph = 0, lt = 0, buf = 0, bph = 0, ncommit = 0;
            const uint32_t ge = static_cast<uint32_t>(GE);
            for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++lt) {
                if (lt >= ge && !mbar_wait(&acce[buf], bph ^ 1u, a.err, kErrWaitEmpty)) {
                    *abort_flag = 1u;
                    break;
                }
                tc_fence_after();
                const uint32_t dj = tmem + buf * static_cast<uint32_t>(a.buf_cols) + js * static_cast<uint32_t>(a.n_slice);
                int r = 0;                                   // chunk within the tap
                for (int i = 0; i < a.nk; ++i) {
                    if (!mbar_wait(&full[st], ph, a.err, kErrWaitFull)) {
                        *abort_flag = 1u;
                        break;
                    }
                    tc_fence_after();
                    const bool s1 = r >= nch0;
                    const uint64_t off = st * stage_units;
                    const uint64_t da = (s1 ? da_s[1] : da_s[0]) + off, db = (s1 ? db_s[1] : db_s[0]) + off;
                    const int n16 = s1 ? n16_s[1] : n16_s[0];
                    for (int kk = 0; kk < n16; ++kk)
                        tc_mma(dj, da + 2u * kk, db + 2u * kk, a.idesc, (i > 0 || kk > 0) ? 1u : 0u);
                    tc_commit(&empty[st]);
                    if (++st == static_cast<uint32_t>(S)) { st = 0; ph ^= 1u; }
                    if (++r == chunks) r = 0;
                }
                tc_commit(&accf[buf]);   // also covers a tile cut short by an abort
                ++ncommit;
                if (++buf == ge) { buf = 0; bph ^= 1u; }
                if (*abort_flag) break;
            }
            // no MMA of this CTA may still run when its TMEM is freed
            for (uint32_t b = 0; b < ge && b < ncommit; ++b) {
                const uint32_t uses = (ncommit - b + ge - 1) / ge;
                mbar_wait(&accf[b], (uses - 1) & 1u, a.err, kErrWaitTail);
            }
        }
    } else {
        // epilogue: warps 4 + 4g .. 7 + 4g drain buffer g (the tiles lt with
        // lt mod GE = g); TMEM lane quarter q = warp % 4
        const int g = (warp - 4) >> 2;
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const uint32_t ge = static_cast<uint32_t>(GE);
        uint32_t lt = static_cast<uint32_t>(g);
        for (int t = blockIdx.x + g * gridDim.x; t < total; t += GE * gridDim.x, lt += ge) {
            const uint32_t buf = lt % ge;
            const bool ok = mbar_wait(&accf[buf], (lt / ge) & 1, a.err, kErrWaitDone);
            tc_fence_after();
            __syncwarp();
            if (!ok || *abort_flag) {
                *abort_flag = 1u;
                break;
            }
            int x0, y, n, n0;
            decode(t, x0, y, n, n0);
            const int x = x0 + row;
            const bool valid = x < a.W;
            const size_t pix = (static_cast<size_t>(n) * a.H + y) * a.W + x;
            const uint32_t tbase = tmem + buf * static_cast<uint32_t>(a.buf_cols) + (static_cast<uint32_t>(q * 32) << 16);
            for (int c = 0; c < a.N_tile; c += 32) {
                const bool two = c + 32 <= a.N_tile;        // uniform: the loads are warp-wide
                const int co0 = n0 + c;
                uint4 mv[4];
                if (valid && co0 < a.N) epi_mask16(a, co0, pix, mv);
                if (valid && two && co0 + 16 < a.N) epi_mask16(a, co0 + 16, pix, mv + 2);
                float v[32];
                if (two) tmem_ld32(tbase + static_cast<uint32_t>(c), v);
                else tmem_ld16(tbase + static_cast<uint32_t>(c), v);
                if (!valid) continue;
                if (co0 < a.N) epilogue16(a, s_bias, v, co0, pix, mv);
                if (two && co0 + 16 < a.N) epilogue16(a, s_bias, v + 16, co0 + 16, pix, mv + 2);
            }
            // this warp's TMEM reads are complete (tcgen05.wait::ld): hand the buffer back
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, static_cast<uint32_t>(a.tmem_cols));
}

// Resident-weight variant for layers whose packed weights fit in shared
// memory (N <= 256): the weights are loaded once per CTA; a tile is R output
// rows x 128 pixels, and each K step is one activation box (input row j,
// column shift dx, channel chunk) that feeds the up to k accumulators of the
// output rows it touches (row r = j - dy with weight tap (dy, dx)), so an
// input row is fetched (R + k - 1) / R times per output row instead of k.
__global__ void __launch_bounds__(kConvMaxThreads) k_conv_res(const __grid_constant__ CUtensorMap ta0,
                                                  const __grid_constant__ CUtensorMap ta1,
                                                  const __grid_constant__ CUtensorMap tb0,
                                                  const __grid_constant__ CUtensorMap tb1, const ConvArgs a) {
    extern __shared__ uint8_t dsm[];
    uint8_t* wsm = align1024(dsm);                        // resident weights
    uint8_t* tiles = wsm + a.w_bytes;                     // ring of activation boxes
    const int S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(tiles + S * a.stage_bytes);
    uint64_t* empty = full + S;
    const int GE = a.epi_groups;                          // accumulator buffers = epilogue warpgroups
    uint64_t* accf = empty + S;
    uint64_t* acce = accf + GE;
    uint64_t* wbar = acce + GE;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(wbar + 1);
    volatile uint32_t* abort_flag = tslot + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ float s_bias[kConvMaxN];                  // the epilogue's bias, read once
    if (a.bias)
        for (int i = threadIdx.x; i < a.N; i += blockDim.x) s_bias[i] = __ldg(&a.bias[i]);

    const int R = a.rows_per_tile, k = a.k, p = k >> 1;
    const int segs = (a.W + 127) >> 7;
    const int groups = (a.H + R - 1) / R;
    const int total = segs * groups * a.Nb;
    const int chunks = a.src[0].nch + (a.nsrc > 1 ? a.src[1].nch : 0);
    const int in_rows = R + k - 1;
    const int steps = in_rows * k * chunks;               // K steps per tile
    const uint32_t acc_cols = static_cast<uint32_t>(a.N_tile);

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], a.n_issue);
        }
        for (int i = 0; i < GE; ++i) {
            mbar_init(&accf[i], a.n_issue);
            mbar_init(&acce[i], 4);
        }
        mbar_init(wbar, 1);
        *abort_flag = 0u;
        mbar_fence_init();
        tma_prefetch(&ta0);
        tma_prefetch(&tb0);
        if (a.nsrc > 1) {
            tma_prefetch(&ta1);
            tma_prefetch(&tb1);
        }
    }
    if (warp == 1) tmem_alloc(tslot, static_cast<uint32_t>(a.tmem_cols));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    auto decode = [&](int t, int& x0, int& y0, int& n) {
        const int xs = t % segs;
        int r = t / segs;
        y0 = (r % groups) * R;
        n = r / groups;
        x0 = xs << 7;
    };
    // K step i of a tile is (input row j, column shift dx, chunk over both
    // sources), chunk fastest: the producer and the MMA warps count them

    if (warp == 0) {
        if (lane == 0) {
            // resident weights: one box per (source, tap, chunk)
            mbar_expect_tx(wbar, a.w_bytes_real);
            for (int s_ = 0; s_ < a.nsrc; ++s_) {
                const ConvSrc& src = a.src[s_];
                const uint32_t tile_bytes = static_cast<uint32_t>(a.N_tile) * src.CW * 2u;
                for (int t = 0; t < k * k; ++t)
                    for (int c = 0; c < src.nch; ++c)
                        tma_load_2d(wsm + a.w_off[s_] + (t * src.nch + c) * tile_bytes, s_ ? &tb1 : &tb0, wbar,
                                    (t * src.nch + c) * src.CW, 0);
            }
            uint32_t it = 0, st = 0, ph = 0;
            const int nch0 = a.src[0].nch;
            for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
                int x0, y0, n;
                decode(t, x0, y0, n);
                int j = 0, dx = 0, rr = 0;                   // K step i = (input row, shift, chunk), counted
                for (int i = 0; i < steps; ++i, ++it) {
                    if (it >= static_cast<uint32_t>(S) && !mbar_wait(&empty[st], ph ^ 1u, a.err, kErrWaitEmpty)) {
                        *abort_flag = 1u;
                        break;
                    }
                    const int s_ = rr < nch0 ? 0 : 1, c = s_ ? rr - nch0 : rr;
                    const ConvSrc& src = a.src[s_];
                    mbar_expect_tx(&full[st], 128u * static_cast<uint32_t>(src.CW) * 2u);
                    tma_load_4d(tiles + st * a.stage_bytes, s_ ? &ta1 : &ta0, &full[st], c * src.CW, x0 + dx - p,
                                y0 - p + j, n);
                    if (++st == static_cast<uint32_t>(S)) { st = 0; ph ^= 1u; }
                    if (++rr == chunks) { rr = 0; if (++dx == k) { dx = 0; ++j; } }
                }
                if (*abort_flag) break;
            }
            const uint32_t issued = it;
            for (uint32_t st = 0; st < static_cast<uint32_t>(S) && st < issued; ++st) {
                const uint32_t last = st + ((issued - 1 - st) / S) * S;
                mbar_wait(&full[st], (last / S) & 1, a.err, kErrWaitTail);
            }
            mbar_wait(wbar, 0, a.err, kErrWaitTail);
        }
    } else if (warp <= 3) {
        // MMA warps 1 .. n_issue: warp 1 + js issues column slice js of every
        // tile.  Descriptors are built once per source (activation stage 0,
        // this slice's weights of tap 0, chunk 0) and advanced by offsets; the
        // K step's (input row, column shift, chunk) is counted, not divided out.
        const uint32_t js = static_cast<uint32_t>(warp - 1);
        if (lane == 0 && warp <= a.n_issue) {
            const uint32_t t0 = smem_u32(tiles), wbase = smem_u32(wsm);
            uint64_t da_s[2], dw_s[2], tb_s[2];
            int n16_s[2], nch_s[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const ConvSrc& src = a.src[q < a.nsrc ? q : 0];
                const uint32_t row = static_cast<uint32_t>(src.CW) * 2u, swz = swz_for_row(row);
                da_s[q] = smem_desc(t0, 16u, 8u * row, swz);
                dw_s[q] = smem_desc(wbase + a.w_off[q < a.nsrc ? q : 0] + js * static_cast<uint32_t>(a.n_slice) * row,
                                    16u, 8u * row, swz);
                tb_s[q] = (static_cast<uint64_t>(a.N_tile) * row) >> 4;   // one weight box, descriptor units
                n16_s[q] = src.CW / 16;
                nch_s[q] = src.nch;
            }
            const uint64_t stage_units = a.stage_bytes >> 4;
            const int nch0 = a.src[0].nch;
            const bool wok = mbar_wait(wbar, 0, a.err, kErrWaitFull);
            if (!wok) *abort_flag = 1u;
            tc_fence_after();
            uint32_t st = 0, ph = 0, lt = 0, buf = 0, bph = 0, ncommit = 0;
            const uint32_t ge = static_cast<uint32_t>(GE);
            for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++lt) {
                if (lt >= ge && !mbar_wait(&acce[buf], bph ^ 1u, a.err, kErrWaitEmpty)) {
                    *abort_flag = 1u;
                    break;
                }
                tc_fence_after();
                const uint32_t d0 = tmem + buf * static_cast<uint32_t>(R) * acc_cols + js * static_cast<uint32_t>(a.n_slice);
                int j = 0, dx = 0, rr = 0;                   // input row, column shift, chunk (all sources)
                for (int i = 0; i < steps; ++i) {
                    if (!mbar_wait(&full[st], ph, a.err, kErrWaitFull)) {
                        *abort_flag = 1u;
                        break;
                    }
                    tc_fence_after();
                    const bool s1 = rr >= nch0;
                    const int c = s1 ? rr - nch0 : rr;
                    const uint64_t da = (s1 ? da_s[1] : da_s[0]) + st * stage_units;
                    const uint64_t dw = s1 ? dw_s[1] : dw_s[0], tb = s1 ? tb_s[1] : tb_s[0];
                    const int n16 = s1 ? n16_s[1] : n16_s[0], nch = s1 ? nch_s[1] : nch_s[0];
                    for (int dy = 0; dy < k; ++dy) {
                        const int r = j - dy;
                        if (r < 0 || r >= R) continue;
                        const uint64_t db = dw + static_cast<uint64_t>((dy * k + dx) * nch + c) * tb;
                        const bool first = (dy == 0 && dx == 0 && rr == 0);
                        const uint32_t dr = d0 + static_cast<uint32_t>(r) * acc_cols;
                        for (int kk = 0; kk < n16; ++kk)
                            tc_mma(dr, da + 2u * kk, db + 2u * kk, a.idesc, (first && kk == 0) ? 0u : 1u);
                    }
                    tc_commit(&empty[st]);
                    if (++st == static_cast<uint32_t>(S)) { st = 0; ph ^= 1u; }
                    if (++rr == chunks) { rr = 0; if (++dx == k) { dx = 0; ++j; } }
                }
                tc_commit(&accf[buf]);
                ++ncommit;
                if (++buf == ge) { buf = 0; bph ^= 1u; }
                if (*abort_flag) break;
            }
            for (uint32_t b = 0; b < ge && b < ncommit; ++b) {
                const uint32_t uses = (ncommit - b + ge - 1) / ge;
                mbar_wait(&accf[b], (uses - 1) & 1u, a.err, kErrWaitTail);
            }
        }
    } else {
        const int g = (warp - 4) >> 2;             // epilogue group = accumulator buffer
        const int q = warp & 3;
        const int prow = q * 32 + lane;
        const uint32_t ge = static_cast<uint32_t>(GE);
        uint32_t lt = static_cast<uint32_t>(g);
        for (int t = blockIdx.x + g * gridDim.x; t < total; t += GE * gridDim.x, lt += ge) {
            const uint32_t buf = lt % ge;
            const bool ok = mbar_wait(&accf[buf], (lt / ge) & 1, a.err, kErrWaitDone);
            tc_fence_after();
            __syncwarp();
            if (!ok || *abort_flag) {
                *abort_flag = 1u;
                break;
            }
            int x0, y0, n;
            decode(t, x0, y0, n);
            const int x = x0 + prow;
            for (int r = 0; r < R; ++r) {
                const int y = y0 + r;
                const bool valid = x < a.W && y < a.H;
                const size_t pix = (static_cast<size_t>(n) * a.H + y) * a.W + x;
                const uint32_t tbase = tmem + (buf * static_cast<uint32_t>(R) + r) * acc_cols +
                                       (static_cast<uint32_t>(q * 32) << 16);
                for (int c = 0; c < a.N_tile; c += 32) {
                    const bool two = c + 32 <= a.N_tile;    // uniform: the loads are warp-wide
                    uint4 mv[4];
                    if (valid && c < a.N) epi_mask16(a, c, pix, mv);
                    if (valid && two && c + 16 < a.N) epi_mask16(a, c + 16, pix, mv + 2);
                    float v[32];
                    if (two) tmem_ld32(tbase + static_cast<uint32_t>(c), v);
                    else tmem_ld16(tbase + static_cast<uint32_t>(c), v);
                    if (!valid) continue;
                    if (c < a.N) epilogue16(a, s_bias, v, c, pix, mv);
                    if (two && c + 16 < a.N) epilogue16(a, s_bias, v + 16, c + 16, pix, mv + 2);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, static_cast<uint32_t>(a.tmem_cols));
}

// Column taps in N (3x3 layers with N <= 64 output channels): tcgen05.mma
// costs about the same per instruction whatever its N, so for narrow layers
// one MMA computes, for the 128 pixels of one input row segment, the products
// with all three column taps at once: D[r][(dx, o)] = sum over (dy, c) of
// in[y + dy - 1][x0 - 1 + r][c] W[o][dy][dx][c] (N = 3 x channels; the three
// row taps accumulate along K).  The output pixel x0 - 1 + r is then
// D[r-1][(0, o)] + D[r][(1, o)] + D[r+1][(2, o)]: the epilogue combines
// neighbouring TMEM lanes with warp shuffles (and a shared-memory exchange
// across warps), and tiles advance by 126 pixels.  Weights are resident in
// shared memory as [dy][chunk][(dx, o)][c].
__global__ void __launch_bounds__(kConvMaxThreads) k_conv_dxn(const __grid_constant__ CUtensorMap ta0,
                                                  const __grid_constant__ CUtensorMap ta1,
                                                  const __grid_constant__ CUtensorMap tb0,
                                                  const __grid_constant__ CUtensorMap tb1, const ConvArgs a) {
    extern __shared__ uint8_t dsm[];
    uint8_t* wsm = align1024(dsm);
    uint8_t* tiles = wsm + a.w_bytes;
    const int S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(tiles + S * a.stage_bytes);
    uint64_t* empty = full + S;
    const int GE = a.epi_groups;                          // accumulator buffers = epilogue warpgroups
    uint64_t* accf = empty + S;
    uint64_t* acce = accf + GE;
    uint64_t* wbar = acce + GE;
    float* xch = reinterpret_cast<float*>(wbar + 1);     // [groups][2 sides][4 warps][16]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(xch + GE * 2 * 2 * 4 * 16);
    volatile uint32_t* abort_flag = tslot + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ float s_bias[kConvMaxN];                  // the epilogue's bias, read once
    __shared__ uint64_t s_da[3][kDxnMaxSteps], s_db[3][kDxnMaxSteps];   // per MMA warp and K step
    __shared__ uint8_t s_nkk[3][kDxnMaxSteps];
    if (a.bias)
        for (int i = threadIdx.x; i < a.N; i += blockDim.x) s_bias[i] = __ldg(&a.bias[i]);

    const int N = a.N;                      // output channels
    const int N3 = 3 * N;                   // MMA N
    const int segs = (a.W + 125) / 126;
    const int total = segs * a.H * a.Nb;
    const int chunks = a.src[0].nch + (a.nsrc > 1 ? a.src[1].nch : 0);
    const int steps = 3 * chunks;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], a.n_issue);
        }
        for (int i = 0; i < GE; ++i) {
            mbar_init(&accf[i], a.n_issue);
            mbar_init(&acce[i], 4);
        }
        mbar_init(wbar, 1);
        *abort_flag = 0u;
        mbar_fence_init();
        tma_prefetch(&ta0);
        tma_prefetch(&tb0);
        if (a.nsrc > 1) {
            tma_prefetch(&ta1);
            tma_prefetch(&tb1);
        }
    }
    if (warp == 1) tmem_alloc(tslot, static_cast<uint32_t>(a.tmem_cols));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    auto decode = [&](int t, int& x0, int& y, int& n) {
        const int xs = t % segs;
        int r = t / segs;
        y = r % a.H;
        n = r / a.H;
        x0 = xs * 126;
    };
    auto step = [&](int i, int& dy, int& s_, int& c) {
        dy = i / chunks;
        const int r = i - dy * chunks;
        s_ = r < a.src[0].nch ? 0 : 1;
        c = s_ ? r - a.src[0].nch : r;
    };

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(wbar, a.w_bytes_real);
            for (int s_ = 0; s_ < a.nsrc; ++s_) {
                const ConvSrc& src = a.src[s_];
                const uint32_t tile_bytes = static_cast<uint32_t>(N3) * src.CW * 2u;
                for (int dy = 0; dy < 3; ++dy)
                    for (int c = 0; c < src.nch; ++c)
                        tma_load_2d(wsm + a.w_off[s_] + (dy * src.nch + c) * tile_bytes, s_ ? &tb1 : &tb0, wbar,
                                    (dy * src.nch + c) * src.CW, 0);
            }
            uint32_t it = 0, st = 0, ph = 0;
            const int nch0 = a.src[0].nch;
            for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
                int x0, y, n;
                decode(t, x0, y, n);
                int dy = 0, rr = 0;                          // K step i = (row tap, chunk), counted
                for (int i = 0; i < steps; ++i, ++it) {
                    if (it >= static_cast<uint32_t>(S) && !mbar_wait(&empty[st], ph ^ 1u, a.err, kErrWaitEmpty)) {
                        *abort_flag = 1u;
                        break;
                    }
                    const int s_ = rr < nch0 ? 0 : 1, c = s_ ? rr - nch0 : rr;
                    const ConvSrc& src = a.src[s_];
                    mbar_expect_tx(&full[st], 128u * static_cast<uint32_t>(src.CW) * 2u);
                    tma_load_4d(tiles + st * a.stage_bytes, s_ ? &ta1 : &ta0, &full[st], c * src.CW, x0 - 1,
                                y + dy - 1, n);
                    if (++st == static_cast<uint32_t>(S)) { st = 0; ph ^= 1u; }
                    if (++rr == chunks) { rr = 0; ++dy; }
                }
                if (*abort_flag) break;
            }
            const uint32_t issued = it;
            for (uint32_t st = 0; st < static_cast<uint32_t>(S) && st < issued; ++st) {
                const uint32_t last = st + ((issued - 1 - st) / S) * S;
                mbar_wait(&full[st], (last / S) & 1, a.err, kErrWaitTail);
            }
            mbar_wait(wbar, 0, a.err, kErrWaitTail);
        }
    } else if (warp <= 3) {
        // MMA warps 1 .. n_issue: warp 1 + js issues column slice js of every tile.
        // The issuing thread shares its scheduler with busy epilogue warps, so
        // its loop is kept short: the descriptors of every K step (A in stage
        // 0, B of this slice) are built once, a stage adds its offset and each
        // 16-channel slice 32 bytes (2 descriptor units).
        const uint32_t js = static_cast<uint32_t>(warp - 1);
        if (lane == 0 && warp <= a.n_issue) {
            uint64_t* da0 = s_da[js];
            uint64_t* db0 = s_db[js];
            uint8_t* nkk = s_nkk[js];
            const uint32_t wbase = smem_u32(wsm);
            const uint32_t tbase_a = smem_u32(tiles);
            for (int i = 0; i < steps; ++i) {
                int dy, s_, c;
                step(i, dy, s_, c);
                const ConvSrc& src = a.src[s_];
                const uint32_t row = static_cast<uint32_t>(src.CW) * 2u;
                const uint32_t swz = swz_for_row(row);
                const uint32_t wt = wbase + a.w_off[s_] + (dy * src.nch + c) * (static_cast<uint32_t>(N3) * row) +
                                    js * static_cast<uint32_t>(a.n_slice) * row;
                da0[i] = smem_desc(tbase_a, 16u, 8u * row, swz);
                db0[i] = smem_desc(wt, 16u, 8u * row, swz);
                nkk[i] = static_cast<uint8_t>(src.CW / 16);
            }
            const uint64_t stage_units = a.stage_bytes >> 4;
            if (!mbar_wait(wbar, 0, a.err, kErrWaitFull)) *abort_flag = 1u;
            tc_fence_after();
            uint32_t st = 0, ph = 0, lt = 0, buf = 0, bph = 0, ncommit = 0;
            const uint32_t ge = static_cast<uint32_t>(GE);
            for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++lt) {
                if (lt >= ge && !mbar_wait(&acce[buf], bph ^ 1u, a.err, kErrWaitEmpty)) {
                    *abort_flag = 1u;
                    break;
                }
                tc_fence_after();
                const uint32_t dj = tmem + buf * static_cast<uint32_t>(a.buf_cols) + js * static_cast<uint32_t>(a.n_slice);
                for (int i = 0; i < steps; ++i) {
                    if (!mbar_wait(&full[st], ph, a.err, kErrWaitFull)) {
                        *abort_flag = 1u;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t da = da0[i] + st * stage_units, db = db0[i];
                    const int n16 = nkk[i];
                    for (int kk = 0; kk < n16; ++kk)
                        tc_mma(dj, da + 2u * kk, db + 2u * kk, a.idesc, (i > 0 || kk > 0) ? 1u : 0u);
                    tc_commit(&empty[st]);
                    if (++st == static_cast<uint32_t>(S)) { st = 0; ph ^= 1u; }
                }
                tc_commit(&accf[buf]);            // also covers a tile cut short by an abort
                ++ncommit;
                if (++buf == ge) { buf = 0; bph ^= 1u; }
                if (*abort_flag) break;
            }
            // no MMA of this CTA may still run when its TMEM is freed: wait for
            // the last commit of every buffer used (commits j < ncommit with
            // j mod ge = b)
            for (uint32_t b = 0; b < ge && b < ncommit; ++b) {
                const uint32_t uses = (ncommit - b + ge - 1) / ge;
                mbar_wait(&accf[b], (uses - 1) & 1u, a.err, kErrWaitTail);
            }
        }
    } else {
        const int g = (warp - 4) >> 2;          // epilogue group = accumulator buffer
        const int q = warp & 3;                 // TMEM lane quarter: rows 32q .. 32q+31
        const int r = q * 32 + lane;
        float* gx0 = xch + g * 256;
        uint32_t xb = 0;
        const uint32_t ge = static_cast<uint32_t>(GE);
        uint32_t lt = static_cast<uint32_t>(g);
        bool dead = false;
        for (int t = blockIdx.x + g * gridDim.x; t < total; t += GE * gridDim.x, lt += ge) {
            const uint32_t buf = lt % ge;
            // A warp that gives up (a wait ran out) stays in the loop without
            // waiting or storing: its group meets at named barriers below, so
            // every warp of the group must take the same number of them.
            if (!dead) {
                const bool ok = mbar_wait(&accf[buf], (lt / ge) & 1, a.err, kErrWaitDone);
                tc_fence_after();
                __syncwarp();
                if (!ok || *abort_flag) {
                    *abort_flag = 1u;
                    dead = true;
                }
            }
            int x0, y, n;
            decode(t, x0, y, n);
            const int x = x0 - 1 + r;
            const bool valid = !dead && r >= 1 && r <= 126 && x < a.W;
            const size_t pix = (static_cast<size_t>(n) * a.H + y) * a.W + (valid ? x : 0);
            const uint32_t tbase = tmem + buf * static_cast<uint32_t>(a.buf_cols) +
                                   (static_cast<uint32_t>(q * 32) << 16);
            for (int c = 0; c < N; c += 16) {
                float v0[16], v1[16], v2[16], o[16];
                tmem_ld16x3(tbase + static_cast<uint32_t>(c), tbase + static_cast<uint32_t>(N + c),
                            tbase + static_cast<uint32_t>(2 * N + c), v0, v1, v2);
                // rows 32q-1 and 32q+32 live in the neighbouring warps; the
                // exchange buffers alternate, so one barrier per chunk suffices
                float* gx = gx0 + (xb & 1u) * 128;
                ++xb;
                if (lane == 31)
#pragma unroll
                    for (int j = 0; j < 16; ++j) gx[(0 * 4 + q) * 16 + j] = v0[j];
                if (lane == 0)
#pragma unroll
                    for (int j = 0; j < 16; ++j) gx[(1 * 4 + q) * 16 + j] = v2[j];
                asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float left = __shfl_up_sync(0xffffffffu, v0[j], 1);
                    float right = __shfl_down_sync(0xffffffffu, v2[j], 1);
                    if (lane == 0) left = q > 0 ? gx[(0 * 4 + q - 1) * 16 + j] : 0.0f;
                    if (lane == 31) right = q < 3 ? gx[(1 * 4 + q + 1) * 16 + j] : 0.0f;
                    o[j] = left + v1[j] + right;
                }
                if (valid) epilogue16(a, s_bias, o, c, pix);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0 && !dead) mbar_arrive(&acce[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, static_cast<uint32_t>(a.tmem_cols));
}

// fp32 master weights -> the column-taps-in-N operand of one source:
// out[(dx, o)][(dy, chunk, c)] = w[o][dy][dx][coff + chunk * CW + c]
// (forward; o < Co) or, for the input gradient, w'[ci][flipped tap][co] with
// (dx, ci) rows.
__global__ void k_pack_dxn(const float* __restrict__ w, int Co, int ci_total, int coff, int C, int CW, int nch,
                           int dgrad, int Nout, __nv_bfloat16* __restrict__ out) {
    const int cols = 3 * nch * CW;
    const long long total = static_cast<long long>(3 * Nout) * cols;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int rr = static_cast<int>(i / cols);
        const int cc = static_cast<int>(i % cols);
        const int dx = rr / Nout, o = rr % Nout;
        const int dy = cc / (nch * CW);
        const int c = cc % (nch * CW);
        float val = 0.0f;
        if (!dgrad) {
            if (c < C) val = w[(static_cast<size_t>(o) * 9 + dy * 3 + dx) * ci_total + coff + c];
        } else {
            // input gradient: rows are input channels o, columns output channels c
            if (c < Co) val = w[(static_cast<size_t>(c) * 9 + (8 - (dy * 3 + dx))) * ci_total + o];
        }
        out[i] = __float2bfloat16_rn(val);
    }
}

// ----------------------------------------------------- weight gradient -----

// Two layouts of the product, both with K = 128 pixels of one row per step:
//  mode 0 (Co >= 128 or k = 1): M = 128 output channels (two 64-channel TMA
//    boxes of dz), N = 64 input channels of one source, one tap row dy per
//    CTA and its k column taps as k accumulators (k shifted boxes of x);
//  mode 1 (Co = 32 or 64, k = 3): M = G = 128 / Co taps x Co channels: the
//    taps are moved onto dz, sum_p dz[p] x[p + o_t] = sum_q dz[q - o_t] x[q],
//    so one unshifted box of x serves G shifted boxes of dz.
__global__ void __launch_bounds__(128) k_wgrad(const __grid_constant__ CUtensorMap tz,
                                               const __grid_constant__ CUtensorMap tx0,
                                               const __grid_constant__ CUtensorMap tx1, const WgradArgs a) {
    extern __shared__ uint8_t dsm[];
    uint8_t* tiles = align1024(dsm);
    const int S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(tiles + S * a.stage_bytes);
    uint64_t* empty = full + S;
    uint64_t* done = empty + S;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int chunks = a.src_chunks[0] + (a.nsrc > 1 ? a.src_chunks[1] : 0);
    int b = blockIdx.x;
    int dy = 0, co_tile = 0, group = 0;
    if (a.mode == 0) {            // blockIdx.x = ((co_tile * chunks) + chunk) * k + dy
        dy = b % a.k;
        b /= a.k;
    }
    const int chunk = b % chunks;
    if (a.mode == 0) co_tile = b / chunks; else group = b / chunks;   // mode 1: (group * chunks) + chunk
    const int s = chunk < a.src_chunks[0] ? 0 : 1;
    const int ch = s ? chunk - a.src_chunks[0] : chunk;
    const int p = a.k >> 1;
    const int per = (a.ksteps + a.splits - 1) / a.splits;
    const int j0 = blockIdx.y * per;
    const int j1 = min(a.ksteps, j0 + per);
    const int nk = max(j1 - j0, 0);
    const int segs = (a.W + 127) >> 7;
    const int G = a.G;                                   // mode 1: taps per CTA
    const uint32_t slice = 128u * static_cast<uint32_t>(a.Co) * 2u;   // mode 1: bytes of one dz box

    // MMA warps 1-3: with three column taps (mode 0, k = 3) warp 1 + dx owns
    // accumulator dx; otherwise the 16-pixel K slices of a box are dealt
    // round-robin to three accumulators that the epilogue adds
    const bool per_dx = (a.mode == 0 && a.k > 1);
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kWgradIssuers);
        }
        mbar_init(done, kWgradIssuers);
        mbar_fence_init();
        tma_prefetch(&tz);
        tma_prefetch(s ? &tx1 : &tx0);
    }
    if (warp == 1) tmem_alloc(tslot, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const CUtensorMap* tx = s ? &tx1 : &tx0;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int st = i % S;
            if (i >= S && !mbar_wait(&empty[st], ((i / S) - 1) & 1, a.err, kErrWaitEmpty)) break;
            const int j = j0 + i;
            const int xs = j % segs;
            const int yy = (j / segs) % a.H;
            const int n = j / (segs * a.H);
            const int x0 = xs << 7;
            uint8_t* sa = tiles + st * a.stage_bytes;
            uint8_t* sb = sa + a.b_region;
            if (a.mode == 0) {
                mbar_expect_tx(&full[st], (2u + static_cast<uint32_t>(a.k)) * 16384u);
                const int co0 = co_tile * 128;
                tma_load_4d(sa, &tz, &full[st], co0, x0, yy, n);
                tma_load_4d(sa + 16384, &tz, &full[st], co0 + 64, x0, yy, n);
                for (int dx = 0; dx < a.k; ++dx)
                    tma_load_4d(sb + dx * 16384, tx, &full[st], ch * 64, x0 + dx - p, yy + dy - p, n);
            } else {
                mbar_expect_tx(&full[st], static_cast<uint32_t>(G) * slice + 16384u);
                for (int g = 0; g < G; ++g) {
                    const int t = group * G + g;
                    // a tap past the last one loads a box wholly outside the image: zeros
                    const int ty = t < a.k * a.k ? t / a.k : 0, tx_ = t < a.k * a.k ? t % a.k : 0;
                    const int ycoord = t < a.k * a.k ? yy - ty + p : -1000000;
                    tma_load_4d(sa + g * slice, &tz, &full[st], 0, x0 - tx_ + p, ycoord, n);
                }
                tma_load_4d(sb, tx, &full[st], ch * 64, x0, yy, n);
            }
            issued = i + 1;
        }
        for (int st = 0; st < S && st < issued; ++st) {
            const int last = st + ((issued - 1 - st) / S) * S;
            mbar_wait(&full[st], (last / S) & 1, a.err, kErrWaitTail);
        }
    } else if (warp >= 1 && warp <= kWgradIssuers && lane == 0) {
        const int j = warp - 1;
        const uint32_t a_row = a.mode == 0 ? 128u : static_cast<uint32_t>(a.Co) * 2u;   // bytes per pixel row of A
        const uint32_t a_swz = a_row == 128u ? kSw128 : kSw64;
        const uint32_t a_lbo = a.mode == 0 ? 16384u : slice;
        for (int i = 0; i < nk; ++i) {
            const int st = i % S;
            if (!mbar_wait(&full[st], (i / S) & 1, a.err, kErrWaitFull)) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(tiles + st * a.stage_bytes);
            const uint32_t sb = sa + a.b_region;
            // this warp's accumulator and K slices: all 8 of tap dx = j, or slices j, j + 3, ...
            const int dx = per_dx ? j : 0;
            const int kk0 = per_dx ? 0 : j, kstep = per_dx ? 1 : kWgradIssuers;
            const uint32_t acc = tmem + static_cast<uint32_t>(j * 64);
            for (int kk = kk0; kk < 8; kk += kstep) {
                // 16 pixels = two 8-row groups
                const uint64_t da = smem_desc(sa + kk * 16u * a_row, a_lbo, 8u * a_row, a_swz);
                const uint64_t db = smem_desc(sb + dx * 16384u + kk * 2048u, 16384u, 1024u, kSw128);
                tc_mma(acc, da, db, a.idesc, (i > 0 || kk > kk0) ? 1u : 0u);
            }
            tc_commit(&empty[st]);
        }
        tc_commit(done);
    }
    __syncwarp();
    const bool ok = mbar_wait(done, 0, a.err, kErrWaitDone) && nk > 0;
    tc_fence_after();
    __syncwarp();

    const int r = warp * 32 + lane;                      // TMEM lane = GEMM row
    const uint32_t tbase = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    const int Cs = a.src_C[s];
    int co, tap_y, tap_x0, ntap;
    if (a.mode == 0) {
        co = co_tile * 128 + r;
        tap_y = dy;
        tap_x0 = 0;
        ntap = a.k;
    } else {
        co = r % a.Co;
        const int t = group * G + r / a.Co;
        tap_y = t / a.k;
        tap_x0 = t % a.k;
        ntap = (t < a.k * a.k) ? 1 : 0;
    }
    const int nacc = per_dx ? a.k : 1;
    for (int dx = 0; dx < nacc; ++dx) {
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tmem_ld16(tbase + static_cast<uint32_t>(dx * 64 + c), v);
            if (!per_dx) {
                // the three K-slice accumulators of the single tap set
                for (int q = 1; q < kWgradIssuers; ++q) {
                    float w[16];
                    tmem_ld16(tbase + static_cast<uint32_t>(q * 64 + c), w);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) v[jj] += w[jj];
                }
            }
            if (!ok || co >= a.Co || ntap == 0) continue;
            const int tx_ = a.mode == 0 ? dx : tap_x0;
            float* dst = a.dW + ((static_cast<size_t>(co) * a.k + tap_y) * a.k + tx_) * a.ci_total + a.src_coff[s];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int ci = ch * 64 + c + jj;
                if (ci < Cs) atomicAdd(dst + ci, v[jj]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, a.tmem_cols);
}

// ---------------------------------------------------------- pointwise -----

namespace {

constexpr int kThreads = 256;

int blocks_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 148 * 64) b = 148 * 64;
    return static_cast<int>(b);
}

__device__ __forceinline__ void load8(const __nv_bfloat16* p, float* f) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i] = __bfloat162float(b[i]);
}

__device__ __forceinline__ void store8(__nv_bfloat16* p, const float* f) {
    __align__(16) __nv_bfloat16 b[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) b[i] = __float2bfloat16_rn(f[i]);
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(b);
}

}  // namespace

// one thread per (pooled pixel, 8 channels)
__global__ void k_maxpool(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int Nb, int H, int W,
                          int C) {
    const int h = H >> 1, w = W >> 1, c8 = C >> 3;
    const long long total = static_cast<long long>(Nb) * h * w * c8;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(i % c8) * 8;
        long long r = i / c8;
        const int xo = static_cast<int>(r % w);
        r /= w;
        const int yo = static_cast<int>(r % h);
        const int n = static_cast<int>(r / h);
        float m[8], f[8];
        load8(x + ((static_cast<size_t>(n) * H + 2 * yo) * W + 2 * xo) * C + c, m);
        for (int q = 1; q < 4; ++q) {
            load8(x + ((static_cast<size_t>(n) * H + 2 * yo + (q >> 1)) * W + 2 * xo + (q & 1)) * C + c, f);
#pragma unroll
            for (int k = 0; k < 8; ++k) m[k] = fmaxf(m[k], f[k]);
        }
        store8(y + ((static_cast<size_t>(n) * h + yo) * w + xo) * C + c, m);
    }
}

// dx = (gradient routed to the first maximum of each 2x2 window) + add
__global__ void k_maxpool_bwd(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ dy,
                              const __nv_bfloat16* __restrict__ add, __nv_bfloat16* __restrict__ dx, int Nb, int H,
                              int W, int C) {
    const int h = H >> 1, w = W >> 1, c8 = C >> 3;
    const long long total = static_cast<long long>(Nb) * h * w * c8;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(i % c8) * 8;
        long long r = i / c8;
        const int xo = static_cast<int>(r % w);
        r /= w;
        const int yo = static_cast<int>(r % h);
        const int n = static_cast<int>(r / h);
        float v[4][8], g[8], best[8];
        int arg[8];
        for (int q = 0; q < 4; ++q)
            load8(x + ((static_cast<size_t>(n) * H + 2 * yo + (q >> 1)) * W + 2 * xo + (q & 1)) * C + c, v[q]);
        load8(dy + ((static_cast<size_t>(n) * h + yo) * w + xo) * C + c, g);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            best[k] = v[0][k];
            arg[k] = 0;
        }
        for (int q = 1; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (v[q][k] > best[k]) {
                    best[k] = v[q][k];
                    arg[k] = q;
                }
        for (int q = 0; q < 4; ++q) {
            const size_t o = ((static_cast<size_t>(n) * H + 2 * yo + (q >> 1)) * W + 2 * xo + (q & 1)) * C + c;
            float out[8], ad[8];
            if (add) load8(add + o, ad);
#pragma unroll
            for (int k = 0; k < 8; ++k) out[k] = (arg[k] == q ? g[k] : 0.0f) + (add ? ad[k] : 0.0f);
            store8(dx + o, out);
        }
    }
}

__global__ void k_upsample(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int Nb, int h, int w,
                           int C) {
    const int H = 2 * h, W = 2 * w, c8 = C >> 3;
    const long long total = static_cast<long long>(Nb) * H * W * c8;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(i % c8) * 8;
        long long r = i / c8;
        const int xx = static_cast<int>(r % W);
        r /= W;
        const int yy = static_cast<int>(r % H);
        const int n = static_cast<int>(r / H);
        const uint4 u = *reinterpret_cast<const uint4*>(x + ((static_cast<size_t>(n) * h + (yy >> 1)) * w + (xx >> 1)) * C + c);
        *reinterpret_cast<uint4*>(y + ((static_cast<size_t>(n) * H + yy) * W + xx) * C + c) = u;
    }
}

__global__ void k_upsample_bwd(const __nv_bfloat16* __restrict__ dy, __nv_bfloat16* __restrict__ dx, int Nb, int h,
                               int w, int C) {
    const int H = 2 * h, W = 2 * w, c8 = C >> 3;
    const long long total = static_cast<long long>(Nb) * h * w * c8;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(i % c8) * 8;
        long long r = i / c8;
        const int xo = static_cast<int>(r % w);
        r /= w;
        const int yo = static_cast<int>(r % h);
        const int n = static_cast<int>(r / h);
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0}, f[8];
        for (int q = 0; q < 4; ++q) {
            load8(dy + ((static_cast<size_t>(n) * H + 2 * yo + (q >> 1)) * W + 2 * xo + (q & 1)) * C + c, f);
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k] += f[k];
        }
        store8(dx + ((static_cast<size_t>(n) * h + yo) * w + xo) * C + c, s);
    }
}

// db[co] += sum over pixels of dz[p][co], with 16-byte loads: a thread sums 8
// channels of its pixels in registers (Co and the stride Cz multiples of 8, dz
// 16-byte aligned), so the reduction is bound by memory rather than by one
// load per element; one f32 atomic per channel per block.
__global__ void k_bias_grad8(const __nv_bfloat16* __restrict__ dz, int Cz, int Co, long long npix, float* db) {
    __shared__ float acc[256 * 8];
    const int chunks = Co / 8;               // 1 .. 32
    const int lanes = 256 / chunks;          // pixels in flight per block
    const int j = threadIdx.x % chunks;
    const int l = threadIdx.x / chunks;
    float s[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (l < lanes)
        for (long long q = static_cast<long long>(blockIdx.x) * lanes + l; q < npix;
             q += static_cast<long long>(gridDim.x) * lanes) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(dz + q * Cz) + j);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
                s[2 * k] += f.x;
                s[2 * k + 1] += f.y;
            }
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[l * Co + 8 * j + k] = (l < lanes) ? s[k] : 0.0f;
    __syncthreads();
    for (int c = threadIdx.x; c < Co; c += blockDim.x) {
        float t = 0.0f;
        for (int k = 0; k < lanes; ++k) t += acc[k * Co + c];
        atomicAdd(&db[c], t);
    }
}

// The same for any Co dividing 256 (the 1-channel output layer): block = 256
// threads over (pixel lane, channel) pairs, one element per load.
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dz, int Cz, int Co, long long npix, float* db) {
    __shared__ float acc[256];
    const int lanes = 256 / Co;              // Co divides 256 or is 1
    const int c = threadIdx.x % Co;
    const int l = threadIdx.x / Co;
    float s = 0.0f;
    if (l < lanes)
        for (long long q = static_cast<long long>(blockIdx.x) * lanes + l; q < npix;
             q += static_cast<long long>(gridDim.x) * lanes)
            s += __bfloat162float(dz[q * Cz + c]);
    acc[threadIdx.x] = (l < lanes) ? s : 0.0f;
    __syncthreads();
    if (threadIdx.x < Co) {
        float t = 0.0f;
        for (int k = 0; k < lanes; ++k) t += acc[k * Co + threadIdx.x];
        atomicAdd(&db[threadIdx.x], t);
    }
}

// Mean squared error of y against t (n values) and its gradient 2 (y - t) / n
// (bf16, written with stride dy_stride; other channels of dy stay zero).
// Per-block partial sums in FP64, then one block adds them in a fixed order.
__global__ void k_mse(const __nv_bfloat16* __restrict__ y, int ys, const __nv_bfloat16* __restrict__ t, long long n,
                      __nv_bfloat16* __restrict__ dy, int ds, double* partials) {
    __shared__ double red[kThreads];
    double s = 0.0;
    const float scale = 2.0f / static_cast<float>(n);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float d = __bfloat162float(y[i * ys]) - __bfloat162float(t[i]);
        s += static_cast<double>(d) * d;
        dy[i * ds] = __float2bfloat16_rn(scale * d);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_mse_final(const double* partials, int nparts, long long n, double* loss) {
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partials[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / static_cast<double>(n);
}

// Adam (Kingma and Ba, Algorithm 1); c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_pack_fwd(const float* __restrict__ w, int Co, int rows, int k, int ci_total, int coff, int C,
                           int CW, int nch, __nv_bfloat16* __restrict__ out) {
    const int kk = k * k, row = kk * nch * CW;
    const long long total = static_cast<long long>(rows) * row;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int co = static_cast<int>(i / row);
        const int r = static_cast<int>(i % row);
        const int tap = r / (nch * CW);
        const int c = r % (nch * CW);
        const float val =
            (co < Co && c < C) ? w[(static_cast<size_t>(co) * kk + tap) * ci_total + coff + c] : 0.0f;
        out[i] = __float2bfloat16_rn(val);
    }
}

// Input-gradient operand: out[ci][t'][co] = w[co][k*k-1-t'][ci]
__global__ void k_pack_dgrad(const float* __restrict__ w, int Co, int k, int ci_total, int rows, int CWz, int nchz,
                             __nv_bfloat16* __restrict__ out) {
    const int kk = k * k, row = kk * nchz * CWz;
    const long long total = static_cast<long long>(rows) * row;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int ci = static_cast<int>(i / row);
        const int r = static_cast<int>(i % row);
        const int tp = r / (nchz * CWz);
        const int co = r % (nchz * CWz);
        const float val =
            (co < Co && ci < ci_total) ? w[(static_cast<size_t>(co) * kk + (kk - 1 - tp)) * ci_total + ci] : 0.0f;
        out[i] = __float2bfloat16_rn(val);
    }
}

__global__ void k_prep(const float* __restrict__ img, int planes, long long hw, float scale, long long npix,
                       __nv_bfloat16* __restrict__ out, int out_C) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < npix;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long n = i / hw, p = i - n * hw;
        const float* src = img + n * planes * hw + p;
        for (int c = 0; c < out_C; ++c) {
            const float v = c < planes ? src[c * hw] * (c == 0 ? scale : 1.0f) : 0.0f;
            out[i * out_C + c] = __float2bfloat16_rn(v);
        }
    }
}

__global__ void k_to_f32(const __nv_bfloat16* __restrict__ x, int stride, long long npix, float scale,
                         float* __restrict__ out) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < npix;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        out[i] = __bfloat162float(x[i * stride]) * scale;
}

// ----------------------------------------------------------- launchers ----

// Each kernel may use the SM's opt-in shared memory (227 KB) less its static arrays.
template <class K>
static cudaError_t allow_dynamic_smem(K kernel) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int total = 227 * 1024;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                total - static_cast<int>(fa.sharedSizeBytes));
}

cudaError_t conv_prepare() {
    cudaError_t e = allow_dynamic_smem(k_conv);
    if (e == cudaSuccess) e = allow_dynamic_smem(k_conv_res);
    if (e == cudaSuccess) e = allow_dynamic_smem(k_conv_dxn);
    if (e == cudaSuccess) e = allow_dynamic_smem(k_wgrad);
    return e;
}

static size_t conv_smem(int stages, uint32_t stage_bytes, int groups = 2) {
    return 1024 + static_cast<size_t>(stages) * stage_bytes + (2 * stages + 2 * groups) * 8 + 16;
}

cudaError_t launch_conv(const CUtensorMap* ta, const CUtensorMap* tb, const ConvArgs& a, cudaStream_t s) {
    const int segs = (a.W + 127) / 128;
    if (a.dxn) {
        const long long total = static_cast<long long>((a.W + 125) / 126) * a.H * a.Nb;
        const int grid = static_cast<int>(std::min<long long>(total, a.grid));
        const size_t smem = 1024 + a.w_bytes + static_cast<size_t>(a.stages) * a.stage_bytes +
                            (2 * a.stages + 2 * a.epi_groups + 1) * 8 + a.epi_groups * 2 * 2 * 4 * 16 * 4 + 16;
        k_conv_dxn<<<grid, 32 * (4 + 4 * a.epi_groups), smem, s>>>(ta[0], ta[a.nsrc > 1 ? 1 : 0], tb[0],
                                                                 tb[a.nsrc > 1 ? 1 : 0], a);
        return cudaGetLastError();
    }
    if (a.rows_per_tile > 0) {
        const long long total = static_cast<long long>(segs) * ((a.H + a.rows_per_tile - 1) / a.rows_per_tile) * a.Nb;
        const int grid = static_cast<int>(std::min<long long>(total, a.grid));
        const size_t smem =
            1024 + a.w_bytes + static_cast<size_t>(a.stages) * a.stage_bytes + (2 * a.stages + 2 * a.epi_groups + 1) * 8 + 16;
        k_conv_res<<<grid, 32 * (4 + 4 * a.epi_groups), smem, s>>>(ta[0], ta[a.nsrc > 1 ? 1 : 0], tb[0],
                                                                 tb[a.nsrc > 1 ? 1 : 0], a);
        return cudaGetLastError();
    }
    const long long total = static_cast<long long>(segs) * a.H * a.Nb * ((a.N + a.N_tile - 1) / a.N_tile);
    const int grid = static_cast<int>(std::min<long long>(total, a.grid));
    k_conv<<<grid, 32 * (4 + 4 * a.epi_groups), conv_smem(a.stages, a.stage_bytes, a.epi_groups), s>>>(
        ta[0], ta[a.nsrc > 1 ? 1 : 0], tb[0],
                                                                 tb[a.nsrc > 1 ? 1 : 0], a);
    return cudaGetLastError();
}

cudaError_t launch_wgrad(const CUtensorMap* tz, const CUtensorMap* tx, const WgradArgs& a, cudaStream_t s) {
    const int chunks = a.src_chunks[0] + (a.nsrc > 1 ? a.src_chunks[1] : 0);
    const int rows = a.mode == 0 ? a.co_tiles * a.k : (a.k * a.k + a.G - 1) / a.G;
    const dim3 grid(rows * chunks, a.splits);
    k_wgrad<<<grid, 128, conv_smem(a.stages, a.stage_bytes), s>>>(*tz, tx[0], tx[a.nsrc > 1 ? 1 : 0], a);
    return cudaGetLastError();
}

cudaError_t launch_maxpool(const __nv_bfloat16* x, __nv_bfloat16* y, int Nb, int H, int W, int C, cudaStream_t s) {
    k_maxpool<<<blocks_for(static_cast<long long>(Nb) * (H / 2) * (W / 2) * (C / 8)), kThreads, 0, s>>>(x, y, Nb, H,
                                                                                                      W, C);
    return cudaGetLastError();
}

cudaError_t launch_maxpool_bwd(const __nv_bfloat16* x, const __nv_bfloat16* dy, const __nv_bfloat16* add,
                               __nv_bfloat16* dx, int Nb, int H, int W, int C, cudaStream_t s) {
    k_maxpool_bwd<<<blocks_for(static_cast<long long>(Nb) * (H / 2) * (W / 2) * (C / 8)), kThreads, 0, s>>>(
        x, dy, add, dx, Nb, H, W, C);
    return cudaGetLastError();
}

cudaError_t launch_upsample(const __nv_bfloat16* x, __nv_bfloat16* y, int Nb, int h, int w, int C, cudaStream_t s) {
    k_upsample<<<blocks_for(static_cast<long long>(Nb) * 4 * h * w * (C / 8)), kThreads, 0, s>>>(x, y, Nb, h, w, C);
    return cudaGetLastError();
}

cudaError_t launch_upsample_bwd(const __nv_bfloat16* dy, __nv_bfloat16* dx, int Nb, int h, int w, int C,
                                cudaStream_t s) {
    k_upsample_bwd<<<blocks_for(static_cast<long long>(Nb) * h * w * (C / 8)), kThreads, 0, s>>>(dy, dx, Nb, h, w,
                                                                                                 C);
    return cudaGetLastError();
}

cudaError_t launch_bias_grad(const __nv_bfloat16* dz, int Cz, int Co, long long npix, float* db, cudaStream_t s) {
    if (Co % 8 == 0 && Co <= 256 && 256 % (Co / 8) == 0 && Cz % 8 == 0 &&
        reinterpret_cast<uintptr_t>(dz) % 16 == 0) {
        const int lanes = 256 / (Co / 8);
        long long b = (npix + lanes - 1) / lanes;
        if (b > 148 * 8) b = 148 * 8;
        if (b < 1) b = 1;
        k_bias_grad8<<<static_cast<int>(b), 256, 0, s>>>(dz, Cz, Co, npix, db);
        return cudaGetLastError();
    }
    const int lanes = 256 / Co;
    long long b = (npix + lanes - 1) / lanes;
    if (b > 148 * 8) b = 148 * 8;
    if (b < 1) b = 1;
    k_bias_grad<<<static_cast<int>(b), 256, 0, s>>>(dz, Cz, Co, npix, db);
    return cudaGetLastError();
}

int mse_parts() { return 148 * 4; }

cudaError_t launch_mse(const __nv_bfloat16* y, int ys, const __nv_bfloat16* t, long long n, __nv_bfloat16* dy,
                       int ds, double* partials, int nparts, double* loss, cudaStream_t s) {
    k_mse<<<nparts, kThreads, 0, s>>>(y, ys, t, n, dy, ds, partials);
    k_mse_final<<<1, kThreads, 0, s>>>(partials, nparts, n, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t s) {
    k_adam<<<blocks_for(n), kThreads, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_pack_fwd(const float* w, int Co, int rows, int k, int ci_total, int coff, int C, int CW, int nch,
                            __nv_bfloat16* out, cudaStream_t s) {
    k_pack_fwd<<<blocks_for(static_cast<long long>(rows) * k * k * nch * CW), kThreads, 0, s>>>(
        w, Co, rows, k, ci_total, coff, C, CW, nch, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_dgrad(const float* w, int Co, int k, int ci_total, int rows, int CWz, int nchz,
                              __nv_bfloat16* out, cudaStream_t s) {
    k_pack_dgrad<<<blocks_for(static_cast<long long>(rows) * k * k * nchz * CWz), kThreads, 0, s>>>(
        w, Co, k, ci_total, rows, CWz, nchz, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_dxn(const float* w, int Co, int ci_total, int coff, int C, int CW, int nch, int dgrad,
                            int Nout, __nv_bfloat16* out, cudaStream_t s) {
    k_pack_dxn<<<blocks_for(static_cast<long long>(3 * Nout) * 3 * nch * CW), kThreads, 0, s>>>(
        w, Co, ci_total, coff, C, CW, nch, dgrad, Nout, out);
    return cudaGetLastError();
}

cudaError_t launch_prep(const float* img, int planes, long long hw, float scale, long long npix,
                        __nv_bfloat16* out, int out_C, cudaStream_t s) {
    k_prep<<<blocks_for(npix), kThreads, 0, s>>>(img, planes, hw, scale, npix, out, out_C);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const __nv_bfloat16* x, int stride, long long npix, float scale, float* out,
                          cudaStream_t s) {
    k_to_f32<<<blocks_for(npix), kThreads, 0, s>>>(x, stride, npix, scale, out);
    return cudaGetLastError();
}

}  // namespace dn
