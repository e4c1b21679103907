// Measured ceiling of the integrator's dominant work: Philox4x32 rounds.
// Every thread runs independent round chains (two 32 x 32 -> 64 multiplies
// and two three-input XORs per round, exactly the round of the integrator's
// generator) at full occupancy with no memory traffic in the loop, so the
// rate it reports is the SM's throughput for that instruction mix.
#include <cuda_runtime.h>

#include "bd_device.cuh"

namespace bdra {
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 512;

__global__ void __launch_bounds__(kProbeThreads, 2)
philox_round_probe(uint32_t* sink, int iters, uint32_t k0, uint32_t k1)
{
    uint4 c[kProbeChains];
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) c[j] = make_uint4(g, (uint32_t)j, g ^ 0x5bd1e995u, (uint32_t)j * 7u);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) {
            uint32_t hi0, lo0, hi1, lo1;
            philox_mulhilo(0xD2511F53u, c[j].x, hi0, lo0);
            philox_mulhilo(0xCD9E8D57u, c[j].z, hi1, lo1);
            c[j] = make_uint4(hi1 ^ c[j].y ^ k0, lo1, hi0 ^ c[j].w ^ k1, lo0);
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc ^= c[j].x ^ c[j].y ^ c[j].z ^ c[j].w;
    sink[g] = acc;
}

// Float32 fused multiply-adds: every thread runs kProbeChains independent
// chains x = fma(x, b, c) with b just below 1 (values stay finite), so the
// rate is the SM's float32 FMA throughput.
__global__ void __launch_bounds__(kProbeThreads, 2)
fma_probe(float* sink, int iters, float b, float c)
{
    float x[kProbeChains];
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) x[j] = (float)(g & 255u) + (float)j;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) x[j] = __fmaf_rn(x[j], b, c);
    }
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc += x[j];
    sink[g] = acc;
}

// Float64 fused multiply-adds, the same way (the FP64 path's unit).
__global__ void __launch_bounds__(kProbeThreads, 2)
dfma_probe(double* sink, int iters, double b, double c)
{
    double x[kProbeChains];
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) x[j] = (double)(g & 255u) + (double)j;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) x[j] = __fma_rn(x[j], b, c);
    }
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc += x[j];
    sink[g] = acc;
}

// Special-function unit: independent chains of approximate reciprocal square
// roots (one MUFU operation each), x = rsqrt(x) + c stays in [1, 2).
__global__ void __launch_bounds__(kProbeThreads, 2)
mufu_probe(float* sink, int iters, float c)
{
    float x[kProbeChains];
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) x[j] = 1.0f + (float)((g + j) & 7u) * 0.125f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) {
            float r;
            asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[j]));
            x[j] = r + c;
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc += x[j];
    sink[g] = acc;
}

// Issue rate of a mixed integer / float32 instruction stream: every thread
// runs kProbeChains independent chains, each iteration two float32 FMAs and
// one three-input logic operation per chain (written as PTX so that each is
// one instruction). The float32 pipe takes two of every three instructions
// and the integer pipe one, neither at its own limit, so the rate is bounded
// by instruction issue (one warp instruction per sub-partition per clock):
// the ceiling of a kernel whose work is a mix of both. Loop control (three
// instructions per 96 counted) is not counted, so the rate errs low by 3%.
__global__ void __launch_bounds__(kProbeThreads, 2)
issue_probe(uint32_t* sink, int iters, float b, float c, uint32_t k)
{
    float x[kProbeChains], y[kProbeChains];
    uint32_t z[kProbeChains];
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) {
        x[j] = (float)(g & 255u) + (float)j;
        y[j] = (float)(g & 127u) - (float)j;
        z[j] = g * 0x9E3779B9u + (uint32_t)j;
    }
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) {
            asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[j]) : "f"(b), "f"(c));
            asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(y[j]) : "f"(b), "f"(c));
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(z[j]) : "r"(k), "r"(g));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc ^= __float_as_uint(x[j]) ^ __float_as_uint(y[j]) ^ z[j];
    sink[g] = acc;
}

// Integer ALU pipe: independent chains of three-input logic operations
// (LOP3, one instruction each, written as PTX), full occupancy.
__global__ void __launch_bounds__(kProbeThreads, 2)
lop3_probe(uint32_t* sink, int iters, uint32_t k)
{
    uint32_t z[kProbeChains];
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) z[j] = g * 0x9E3779B9u + (uint32_t)j;
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j)
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(z[j]) : "r"(k), "r"(g));
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc ^= z[j];
    sink[g] = acc;
}

// Times `launch(iters)` on `stream` after a warm-up launch (iters 256) and
// returns the shortest duration of three launches in ms (0 on failure).
template <typename F>
float probe_time(cudaStream_t st, F launch, int iters)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        launch(256);
        for (int rep = 0; rep < 3; ++rep) {      // a ceiling: the fastest of three launches
            float t = 0.0f;
            cudaEventRecord(e0, st);
            launch(iters);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
                cudaGetLastError() != cudaSuccess) {
                ms = 0.0f;
                break;
            }
            if (rep == 0 || t < ms) ms = t;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
    return ms;
}

}  // namespace
}  // namespace bdra

using namespace bdra;

namespace {
// Device SM count (0 on failure).
int probe_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms;
}
}  // namespace

extern "C" bd_status bd_probe_fp64_fma(void* stream, double* flops_per_s)
{
    if (!flops_per_s) return BD_E_INVALID;
    *flops_per_s = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = probe_sms();
    if (!sms) return BD_E_CUDA;
    const int blocks = 2 * sms, iters = 1024;
    double* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(double) * (size_t)blocks * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return BD_E_OOM;
    }
    const float ms = probe_time(st, [&](int n) {
        dfma_probe<<<blocks, kProbeThreads, 0, st>>>(sink, n, 0.9999999999999999, 1e-3);
    }, iters);
    cudaFree(sink);
    cudaGetLastError();
    if (!(ms > 0.0f)) return BD_E_CUDA;
    *flops_per_s = 2.0 * (double)blocks * kProbeThreads * iters * kProbeChains / (ms * 1e-3);
    return BD_OK;
}

extern "C" bd_status bd_probe_mufu(void* stream, double* ops_per_s)
{
    if (!ops_per_s) return BD_E_INVALID;
    *ops_per_s = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = probe_sms();
    if (!sms) return BD_E_CUDA;
    const int blocks = 2 * sms, iters = 4096;
    float* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(float) * (size_t)blocks * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return BD_E_OOM;
    }
    const float ms = probe_time(st, [&](int n) {
        mufu_probe<<<blocks, kProbeThreads, 0, st>>>(sink, n, 0.75f);
    }, iters);
    cudaFree(sink);
    cudaGetLastError();
    if (!(ms > 0.0f)) return BD_E_CUDA;
    *ops_per_s = (double)blocks * kProbeThreads * iters * kProbeChains / (ms * 1e-3);
    return BD_OK;
}

extern "C" bd_status bd_probe_fp32_fma(void* stream, double* flops_per_s)
{
    if (!flops_per_s) return BD_E_INVALID;
    *flops_per_s = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return BD_E_CUDA;
    }
    const int blocks = 2 * sms, iters = 16384;
    float* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(float) * (size_t)blocks * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return BD_E_OOM;
    }
    const float ms = probe_time(st, [&](int n) {
        fma_probe<<<blocks, kProbeThreads, 0, st>>>(sink, n, 0.99999994f, 1e-3f);
    }, iters);
    cudaFree(sink);
    cudaGetLastError();
    if (!(ms > 0.0f)) return BD_E_CUDA;
    *flops_per_s = 2.0 * (double)blocks * kProbeThreads * iters * kProbeChains / (ms * 1e-3);
    return BD_OK;
}

extern "C" bd_status bd_probe_issue(void* stream, double* lane_instr_per_s)
{
    if (!lane_instr_per_s) return BD_E_INVALID;
    *lane_instr_per_s = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = probe_sms();
    if (!sms) return BD_E_CUDA;
    const int blocks = 2 * sms, iters = 8192;
    uint32_t* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(uint32_t) * (size_t)blocks * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return BD_E_OOM;
    }
    const float ms = probe_time(st, [&](int n) {
        issue_probe<<<blocks, kProbeThreads, 0, st>>>(sink, n, 0.99999994f, 1e-3f, 0x5bd1e995u);
    }, iters);
    cudaFree(sink);
    cudaGetLastError();
    if (!(ms > 0.0f)) return BD_E_CUDA;
    *lane_instr_per_s = 3.0 * (double)blocks * kProbeThreads * iters * kProbeChains / (ms * 1e-3);
    return BD_OK;
}

extern "C" bd_status bd_probe_int_alu(void* stream, double* ops_per_s)
{
    if (!ops_per_s) return BD_E_INVALID;
    *ops_per_s = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = probe_sms();
    if (!sms) return BD_E_CUDA;
    const int blocks = 2 * sms, iters = 8192;
    uint32_t* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(uint32_t) * (size_t)blocks * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return BD_E_OOM;
    }
    const float ms = probe_time(st, [&](int n) {
        lop3_probe<<<blocks, kProbeThreads, 0, st>>>(sink, n, 0x5bd1e995u);
    }, iters);
    cudaFree(sink);
    cudaGetLastError();
    if (!(ms > 0.0f)) return BD_E_CUDA;
    *ops_per_s = (double)blocks * kProbeThreads * iters * kProbeChains / (ms * 1e-3);
    return BD_OK;
}

extern "C" bd_status bd_probe_philox_rounds(void* stream, double* rounds_per_s)
{
    if (!rounds_per_s) return BD_E_INVALID;
    *rounds_per_s = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return BD_E_CUDA;
    }
    const int blocks = 2 * sms, iters = 4096;
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bd_status s = BD_OK;
    float ms = 0.0f;
    if (cudaMalloc((void**)&sink, sizeof(uint32_t) * (size_t)blocks * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return BD_E_OOM;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = BD_E_CUDA;
    if (s == BD_OK) {
        philox_round_probe<<<blocks, kProbeThreads, 0, st>>>(sink, 256, 1u, 2u);    // warm-up
        cudaEventRecord(e0, st);
        philox_round_probe<<<blocks, kProbeThreads, 0, st>>>(sink, iters, 1u, 2u);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess || !(ms > 0.0f))
            s = BD_E_CUDA;
    }
    if (s == BD_OK)
        *rounds_per_s = (double)blocks * kProbeThreads * iters * kProbeChains / (ms * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaGetLastError();
    return s;
}
