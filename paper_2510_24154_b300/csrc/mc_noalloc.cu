// Dose statistics for callers that may not allocate device memory.
//
// mc_get_dose works inside a context that owns cudaMalloc'd scratch.  Some
// callers cannot allocate after start-up: a QA service whose framework
// allocator has already reserved the GPU's memory, or medical software whose
// rules forbid run-time allocation because it can fail or stall at an
// unpredictable moment.  mc_dose_stats_noalloc computes the same per-pixel
// dose, batch sigma and mean relative uncertainty from a tally the caller
// holds, with its scratch (batch counts, the image maximum, per-block partial
// sums) in a fixed array that lives in this file.
#include <cstdio>
#include <mutex>

#include "archer_epid.h"
#include "mc_aux.h"

namespace {

constexpr int kMaxBatches = 1024;
constexpr int kMaxPixels = 1 << 22;                 // 2048 x 2048
constexpr int kBlock = 256;                         // block size of the statistics kernels
constexpr int kMaxParts = kMaxPixels / kBlock;
constexpr size_t kOffNb = 0;                                        // double[kMaxBatches]
constexpr size_t kOffMax = kOffNb + sizeof(double) * kMaxBatches;   // unsigned long long
constexpr size_t kOffSum = kOffMax + 256;                           // double[kMaxParts]
constexpr size_t kOffCnt = kOffSum + sizeof(double) * kMaxParts;    // unsigned int[kMaxParts]
constexpr size_t kScratchBytes = kOffCnt + sizeof(unsigned int) * kMaxParts;
// 8,192 (batch counts) + 256 (maximum) + 131,072 (partial sums) + 65,536 (partial counts)
static_assert(kScratchBytes == 205056, "the documented scratch size must follow the layout");

// Every GPU that loads the library keeps this array until the process exits.
// Host code may not use its name as an address; set-up below asks the runtime
// for the device address.  The address is looked up once per device and kept:
// after cudaDeviceReset (or anything else that destroys the device's primary
// context) it is stale, so this entry point must not be called again in that
// process after such a reset.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {};

// Batch counts for history ids 0 .. n-1 (id mod B), written into the scratch.
__global__ void k_batch_counts(double* nb, int B, unsigned long long n) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) nb[b] = static_cast<double>(n / B + (static_cast<unsigned long long>(b) < n % B ? 1ull : 0ull));
}

}  // namespace

extern "C" mc_status mc_dose_stats_noalloc(const uint64_t* tally, int npx, int npy, int n_batches,
                                           uint64_t n_histories, double pixel_mass_kg, double* dose, double* sigma,
                                           double* u, void* stream) {
    if (!tally || !dose || npx < 1 || npy < 1 || n_batches < 2 || n_histories == 0 || !(pixel_mass_kg > 0.0))
        return MC_ERR_ARG;
    if (static_cast<long long>(npx) * npy > kMaxPixels || n_batches > kMaxBatches) {
        std::fprintf(stderr, "mc_dose_stats_noalloc: image of %d x %d pixels or %d batches exceeds the limit "
                             "of %d pixels and %d batches\n", npx, npy, n_batches, kMaxPixels, kMaxBatches);
        return MC_ERR_ARG;
    }
    if (u && !sigma) return MC_ERR_ARG;
    if (n_histories < static_cast<uint64_t>(n_batches)) {
        // a batch without histories has no mean: sigma and u would be NaN
        std::fprintf(stderr, "mc_dose_stats_noalloc: %llu histories cannot fill %d batches (need at least one "
                             "history per batch)\n", static_cast<unsigned long long>(n_histories), n_batches);
        return MC_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MC_ERR_CUDA;
    unsigned char* base;
    {
        // first call on this device: look up the array's device address
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MC_ERR_CUDA;
            g_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* nb = reinterpret_cast<double*>(base + kOffNb);
    unsigned long long* max_bits = reinterpret_cast<unsigned long long*>(base + kOffMax);
    double* part_sum = reinterpret_cast<double*>(base + kOffSum);
    unsigned int* part_cnt = reinterpret_cast<unsigned int*>(base + kOffCnt);
    k_batch_counts<<<(n_batches + 127) / 128, 128, 0, s>>>(nb, n_batches, n_histories);
    if (cudaGetLastError() != cudaSuccess) return MC_ERR_CUDA;
    // launch_dose clears the maximum before use, so the previous call's value never leaks in
    const int npix = npx * npy;
    if (mc::launch_dose(reinterpret_cast<const unsigned long long*>(tally), npix, n_batches, nb,
                        static_cast<double>(n_histories), 1.602176634e-13 / pixel_mass_kg, dose, sigma, max_bits,
                        part_sum, part_cnt, u, s) != cudaSuccess)
        return MC_ERR_CUDA;
    return MC_OK;
}
