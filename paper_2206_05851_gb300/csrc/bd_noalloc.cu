// Event compaction that allocates nothing (bd_compact_events_noalloc).
//
// Same output as the event list of bd_detect_events, computed from
// caller-supplied kinetic arrays. The per-block counts and offsets it needs
// live in a fixed file-scope device array instead of memory from cudaMalloc,
// so the call can be made by code that may not allocate device memory.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/bdra.h"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kMaxBlocks = BD_NOALLOC_MAX_SPRINGS / kThreads;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: block counts, then offsets, and
// the total at index [n_blocks]. Held by every device that loads the library
// until the process exits.
static __device__ __align__(256) int64_t g_event_scratch[kMaxBlocks + 1];

std::mutex g_mutex;
int64_t* g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ int count_events(int64_t m, int64_t M, const int64_t* first_thr,
                                            const int64_t* first_bell)
{
    int n = 0;
    for (int q = 0; q < 3; ++q) n += (first_thr[q * M + m] >= 0) + (first_bell[q * M + m] >= 0);
    return n;
}

// Exclusive scan of one value per thread over the block; *total = block sum.
__device__ __forceinline__ int block_scan(int v, int* total)
{
    __shared__ int warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < kThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const int before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void noalloc_count_kernel(int64_t M, const int64_t* first_thr,
                                     const int64_t* first_bell, int64_t* scratch)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = m < M ? count_events(m, M, first_thr, first_bell) : 0;
    int total;
    block_scan(v, &total);
    if (threadIdx.x == 0) scratch[blockIdx.x] = total;
}

__global__ void noalloc_scan_kernel(int64_t* scratch, int n_blocks, int64_t* n_out)
{
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n_blocks; base += kThreads) {
        const int j = base + threadIdx.x;
        const int v = j < n_blocks ? (int)scratch[j] : 0;
        int total;
        const int before = block_scan(v, &total);
        if (j < n_blocks) scratch[j] = carry + before;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[n_blocks] = carry;
        *n_out = carry;
    }
}

__global__ void noalloc_write_kernel(int64_t M, const int64_t* first_thr,
                                     const int64_t* first_bell, const int64_t* spring_offsets,
                                     int n_chains, const int64_t* scratch, bd_event* out,
                                     int64_t capacity)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = m < M ? count_events(m, M, first_thr, first_bell) : 0;
    int total;
    const int before = block_scan(v, &total);
    if (m >= M || v == 0) return;
    int lo = 0, hi = n_chains - 1;     // chain c with spring_offsets[c] <= m
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (spring_offsets[mid] <= m) lo = mid; else hi = mid - 1;
    }
    int64_t pos = scratch[blockIdx.x] + before;
    for (int q = 0; q < 3; ++q) {
        for (int kind = 0; kind < 2; ++kind) {
            const int64_t st = kind == 0 ? first_thr[q * M + m] : first_bell[q * M + m];
            if (st < 0) continue;
            if (pos < capacity) {
                bd_event e;
                e.chain = lo;
                e.spring = (int32_t)(m - spring_offsets[lo]);
                e.criterion = q;
                e.kind = kind;
                e.step = st;
                out[pos] = e;
            }
            ++pos;
        }
    }
}

// Device address of g_event_scratch on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(int64_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_event_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<int64_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" bd_status bd_compact_events_noalloc(const int64_t* first_thr,
                                               const int64_t* first_bell, int64_t n_springs,
                                               const int64_t* spring_offsets, int32_t n_chains,
                                               bd_event* out, int64_t capacity, int64_t* n_out,
                                               void* stream)
{
    if (!first_thr || !first_bell || !spring_offsets || !n_out) return BD_E_INVALID;
    if (n_chains < 1 || n_springs < 0 || capacity < 0 || (capacity > 0 && !out))
        return BD_E_INVALID;
    if (n_springs > BD_NOALLOC_MAX_SPRINGS) return BD_E_CAPACITY;
    int64_t* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BD_E_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n_blocks = (int)((n_springs + kThreads - 1) / kThreads);
    if (n_blocks > 0)
        noalloc_count_kernel<<<n_blocks, kThreads, 0, st>>>(n_springs, first_thr, first_bell,
                                                           scratch);
    noalloc_scan_kernel<<<1, kThreads, 0, st>>>(scratch, n_blocks, n_out);
    if (n_blocks > 0)
        noalloc_write_kernel<<<n_blocks, kThreads, 0, st>>>(n_springs, first_thr, first_bell,
                                                           spring_offsets, n_chains, scratch,
                                                           out, capacity);
    e = cudaGetLastError();
    return e == cudaSuccess ? BD_OK : BD_E_CUDA;
}
