// Arithmetic peak probes: measured denominators for the transport kernels'
// ALU roofline (the copy-bandwidth and bf16 GEMM peaks say nothing about the
// FP32 pipe, the transcendental unit or instruction issue).
//
// Each probe runs independent dependency chains of one instruction class in
// every thread of a full-occupancy grid (4 CTAs of 256 threads per SM), long
// enough (a few milliseconds) that launch overhead is negligible, and counts
// the instructions its source issues: 8 chains x 16 unrolled steps per loop
// pass.  The hardware instruction counters agree with these counts
// instruction class by instruction class; the loop's branch (one instruction
// per 128 counted) is left out, so the rates are slight underestimates.
#include <cuda_runtime.h>
#include <stdint.h>

#include "archer_epid.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

// FP32 fused multiply-add, scalar form: x <- x*m + c converges to c/(1-m).
__global__ void __launch_bounds__(kThreads) k_probe_ffma(float* out, int iters, float m, float c) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + 1e-3f * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], m, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP32 fused multiply-add on register pairs (PTX fma.rn.f32x2, sm_100 and
// later): one instruction, two lanes' worth of FMAs.
__global__ void __launch_bounds__(kThreads) k_probe_ffma2(float* out, int iters, float m, float c) {
    unsigned long long x[kChains];
    unsigned long long mm, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(mm) : "f"(m));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        const float a = 1.0f + 1e-3f * (threadIdx.x + i), b = a + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[i]) : "f"(a), "f"(b));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(mm), "l"(cc));
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x[i]));
        s += a + b;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Transcendental unit: alternating base-2 exponential and logarithm
// (ex2.approx / lg2.approx, the forms the fast-math transport uses), so each
// chain returns to its start value instead of overflowing.
__global__ void __launch_bounds__(kThreads) k_probe_mufu(float* out, int iters) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 0.25f + 1e-3f * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; u += 2) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
                asm("lg2.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Integer ALU: add and exclusive-or chains (the Philox rounds' and the
// table indexing's instruction classes).
__global__ void __launch_bounds__(kThreads) k_probe_int(float* out, int iters, uint32_t k1, uint32_t k2) {
    uint32_t x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 2654435761u + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; u += 2) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                x[i] ^= k1;
                x[i] += k2 + i;
            }
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = __uint_as_float(s & 0x3fffffffu);
}

// Issue: FP32 FMAs and integer operations interleaved, two pipes fed from one
// instruction stream.  The integer keys are run-time values: adding the
// unrolled step index instead lets the compiler drop or fold some adds.
__global__ void __launch_bounds__(kThreads) k_probe_mix(float* out, int iters, float m, float c, uint32_t k1,
                                                        uint32_t k2) {
    float x[kChains / 2];
    uint32_t y[kChains / 2];
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) {
        x[i] = 1.0f + 1e-3f * (threadIdx.x + i);
        y[i] = threadIdx.x * 2654435761u + i;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kChains / 2; ++i) {
                x[i] = fmaf(x[i], m, c);
                y[i] = (y[i] ^ k1) + k2;
            }
        }
    }
    float s = 0.0f;
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) {
        s += x[i];
        t ^= y[i];
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s + (float)(t & 0xffu);
}

}  // namespace

extern "C" mc_status mc_probe_alu_peaks(int device, int repeats, mc_alu_peaks* res) {
    if (!res || repeats < 1 || repeats > 100) return MC_ERR_ARG;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return MC_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return MC_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid = sms * kCtasPerSm;
    const double threads = (double)grid * kThreads;
    float* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mc_status rc = MC_OK;
    if (cudaMalloc(&out, sizeof(float) * (size_t)grid * kThreads) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = MC_ERR_CUDA;
    }
    // best time over `repeats` launches after one untimed launch
    auto best_ms = [&](auto launch) -> double {
        launch();
        double best = 1e30;
        for (int r = 0; r < repeats; ++r) {
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) best = ms;
        }
        return cudaGetLastError() == cudaSuccess ? best : -1.0;
    };
    const double per_pass = (double)kChains * kUnroll;
    if (rc == MC_OK) {
        const int it_fma = 8192, it_mufu = 1024, it_int = 4096;
        const double t_fma = best_ms([&] { k_probe_ffma<<<grid, kThreads, 0, st>>>(out, it_fma, 0.9999f, 1e-4f); });
        const double t_fma2 = best_ms([&] { k_probe_ffma2<<<grid, kThreads, 0, st>>>(out, it_fma, 0.9999f, 1e-4f); });
        const double t_mufu = best_ms([&] { k_probe_mufu<<<grid, kThreads, 0, st>>>(out, it_mufu); });
        const double t_int = best_ms([&] { k_probe_int<<<grid, kThreads, 0, st>>>(out, it_int, 0x9E3779B9u, 7u); });
        const double t_mix = best_ms([&] { k_probe_mix<<<grid, kThreads, 0, st>>>(out, it_fma, 0.9999f, 1e-4f, 0x9E3779B9u,
                                                                                  7u); });
        if (t_fma <= 0 || t_fma2 <= 0 || t_mufu <= 0 || t_int <= 0 || t_mix <= 0) {
            rc = MC_ERR_CUDA;
        } else {
            const double n_fma = threads * it_fma * per_pass;    // FMA instructions (per thread, summed)
            res->ffma_tflops = 2.0 * n_fma / (t_fma * 1e-3) / 1e12;
            res->ffma2_tflops = 4.0 * n_fma / (t_fma2 * 1e-3) / 1e12;
            res->mufu_tops = threads * it_mufu * per_pass / (t_mufu * 1e-3) / 1e12;
            // the int probe issues two instructions (xor, add) per chain and pair of steps
            res->int_tinst = threads * it_int * per_pass / (t_int * 1e-3) / 1e12;
            // the mixed probe: per chain and step one FMA, one xor, one add
            res->mix_tinst = threads * it_fma * (kUnroll * (kChains / 2) * 3.0) / (t_mix * 1e-3) / 1e12;
            res->sm_count = sms;
            res->ms_total = t_fma + t_fma2 + t_mufu + t_int + t_mix;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    cudaSetDevice(prev);
    return rc;
}
