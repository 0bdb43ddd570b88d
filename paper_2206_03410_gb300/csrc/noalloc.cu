// nrr_align_energy_noalloc: the alignment term of the energy and the
// surrogate weights from closest-point distances, for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden,
// for example a tracking loop that works only from memory it preallocated
// (real-time budgets), a host framework whose allocator owns every device
// allocation, or work enqueued while another component is capturing a CUDA
// graph. Such callers cannot create an nrr context (which allocates), so this
// entry point takes only caller-owned input and output buffers and keeps its
// scratch (the per-CTA partial sums of the reduction and the completion
// counter) in a fixed static device array.
//
// The scratch array is 64 KiB of file-scope __device__ memory (kScratchBytes);
// every GPU that loads the library holds it until the process exits.
// Its device address is looked up once per device (cudaGetSymbolAddress with
// that device current) on the first call made on that device. Every call
// shares the array and it keeps the last call's contents, so the completion
// counter is cleared at the start of each call; calls that overlap on the GPU
// (different streams, or host threads on the same device) race on it and
// must be serialised by the caller.
#include <mutex>

#include "nrr_device.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItemsPerThread = 16;
constexpr int kPointsPerBlock = kThreads * kItemsPerThread;   // 4096
constexpr size_t kScratchBytes = 64 * 1024;
constexpr size_t kPartialOffset = 256;                          // after the counter
constexpr int kMaxBlocks = (int)((kScratchBytes - kPartialOffset) / sizeof(double));   // 8160
constexpr int64_t kMaxPoints = (int64_t)kMaxBlocks * kPointsPerBlock;                 // 33,423,360
constexpr int kMaxDevices = 64;

// counter at offset 0, per-CTA partial sums from offset 256
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::once_flag g_once[kMaxDevices];
void* g_scratch_ptr[kMaxDevices] = {nullptr};
cudaError_t g_scratch_err[kMaxDevices] = {cudaSuccess};

__global__ void __launch_bounds__(kThreads)
align_energy_kernel(const float* __restrict__ d2, int64_t P, float ia, float* __restrict__ wa,
                    double* __restrict__ E_out, unsigned char* scratch) {
    __shared__ double sh[kThreads / 32];
    __shared__ int s_last;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* partials = reinterpret_cast<double*>(scratch + kPartialOffset);
    const int64_t base = (int64_t)blockIdx.x * kPointsPerBlock;
    double e = 0.0;
#pragma unroll 4
    for (int k = 0; k < kItemsPerThread; ++k) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < P) {
            const float x = d2[i] * ia;
            e += (double)(-expm1f(-x));        // Welsch's function psi_nu_a (Sec. 3.2)
            wa[i] = expf(-x) * ia;             // weight of the quadratic surrogate
        }
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w];
        partials[blockIdx.x] = s;
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kThreads) s += __ldcg(partials + b);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
        *E_out = t;
        *counter = 0u;
    }
}

}  // namespace

extern "C" nrr_status nrr_align_energy_noalloc(const float* d2, int64_t P, double nu_a, float* w_a,
                                               double* E_align, void* cuda_stream) {
    if (!d2 || !w_a || !E_align) return nrr_set_global_error(NRR_E_INVALID, "nrr_align_energy_noalloc: NULL buffer");
    if (P < 1 || P > kMaxPoints)   // the scratch holds kMaxBlocks partial sums
        return nrr_set_global_error(NRR_E_INVALID,
                                    "nrr_align_energy_noalloc: P must be in 1..33423360 (static scratch limit)");
    if (!(nu_a > 0) || !(nu_a < INFINITY))
        return nrr_set_global_error(NRR_E_INVALID, "nrr_align_energy_noalloc: nu_a must be positive and finite");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nrr_set_global_error(NRR_E_CUDA, "nrr_align_energy_noalloc: no usable current device");
    std::call_once(g_once[dev], [dev]() {
        void* p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_scratch_ptr[dev] = p;
    });
    if (g_scratch_err[dev] != cudaSuccess || !g_scratch_ptr[dev])
        return nrr_set_global_error(NRR_E_CUDA, "nrr_align_energy_noalloc: cudaGetSymbolAddress failed");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* scratch = (unsigned char*)g_scratch_ptr[dev];
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned), s) != cudaSuccess)
        return nrr_set_global_error(NRR_E_CUDA, "nrr_align_energy_noalloc: clearing the counter failed");
    const int grid = (int)((P + kPointsPerBlock - 1) / kPointsPerBlock);
    const float ia = (float)(1.0 / (2.0 * nu_a * nu_a));
    align_energy_kernel<<<grid, kThreads, 0, s>>>(d2, P, ia, w_a, E_align, scratch);
    if (cudaGetLastError() != cudaSuccess)
        return nrr_set_global_error(NRR_E_CUDA, "nrr_align_energy_noalloc: kernel launch failed");
    return NRR_OK;
}
