// probe.cu -- short measurements of this GPU's compute peaks for the roofline terms the kernels are
// bound by: binary32 FMA, the 5th-generation tensor cores on binary16 operands with binary32
// accumulation (tcgen05.mma kind::f16, M = 128, N = 256, K = 16, operands in shared memory), and
// shared-memory 32-bit reductions (conflict-free, random addresses, binary32 adds).  Each is one
// kernel launch of a fixed amount of work on every SM, timed with CUDA events on the given stream.
#include <cuda_runtime.h>

#include <cstring>

#include "enufft.h"
#include "internal.h"
#include "tc.cuh"

namespace enufft {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kFmaIters = 4096;
constexpr int kRedIters = 1024;
constexpr int kMmaIters = 4096;
constexpr unsigned kMmaWait = 1u << 17;
constexpr int kMmaPadSmem = 120 * 1024;   // dynamic shared memory that keeps one probe CTA per SM

__global__ void __launch_bounds__(kProbeThreads, 2) probe_fma_kernel(float* sink, float seed) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x + k;
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __fmaf_rn(a[k], 0.99999f, 0.5f);
    }
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += a[k];
    if (t == 1234.5f) sink[threadIdx.x] = t;   // never true; keeps the chains live
}

__device__ __forceinline__ unsigned probe_hash(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// MODE 0: red.shared.add.u32, lane l of warp w always in bank l; 1: random words; 2: red.shared.add.f32,
// bank = lane.  16384 words of shared memory; every offset is taken modulo that size.
template <int MODE>
__global__ void __launch_bounds__(kProbeThreads, 2) probe_red_kernel(float* sink) {
    __shared__ unsigned s[16384];
    for (int i = threadIdx.x; i < 16384; i += kProbeThreads) s[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned off[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        off[k] = MODE == 1 ? probe_hash(blockIdx.x * 7919u + threadIdx.x * 8u + k) % 16384u
                           : (unsigned)(((warp * 8 + k) * 32 + lane) % 16384);
    const unsigned base = (unsigned)__cvta_generic_to_shared(s);
    for (int it = 0; it < kRedIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (MODE == 2)
                asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(base + off[k] * 4), "f"(1.0f) : "memory");
            else
                asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(base + off[k] * 4), "r"(it + k) : "memory");
        }
    }
    __syncthreads();
    if (s[threadIdx.x] == 0xdeadbeefu) sink[threadIdx.x] = 1.0f;
}

// One CTA per SM: one thread issues kMmaIters back-to-back MMAs (128 x 256 x 16, binary16 operands
// from zeroed shared memory, binary32 accumulator in tensor memory), commits them to an mbarrier and
// waits for it with a bounded wait; ok[blockIdx] = 1 when the MMAs completed.
__global__ void __launch_bounds__(128, 1) probe_mma_kernel(int* ok) {
    constexpr int M = 128, N = 256, KK = 16;
    constexpr unsigned kA = M * KK * 2, kB = N * KK * 2;   // operand bytes of one MMA
    __shared__ __align__(1024) unsigned char ops[kA + kB];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (int)(kA + kB) / 16; i += 128) reinterpret_cast<uint4*>(ops)[i] = make_uint4(0, 0, 0, 0);
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_addr(&tbase), 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_addr(&bar), 1);
        tc::mbar_init_fence();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const unsigned tmem = tbase;
    if (tid == 0) {
        // MN-major, no swizzle: 8 x 8 core matrices of 128 B, feature blocks 128 B apart, the two
        // K octets of the MMA M * 16 (A) or N * 16 (B) bytes apart
        const unsigned sa = tc::smem_addr(ops), sb = sa + kA;
        const uint64_t ad = tc::smem_desc(sa, M * 16, 128), bd = tc::smem_desc(sb, N * 16, 128);
        const unsigned idesc = tc::idesc_f16_f32_mn(M, N);
        for (int it = 0; it < kMmaIters; ++it) tc::mma_f16(tmem, ad, bd, idesc, it > 0 ? 1u : 0u);
        tc::mma_commit(tc::smem_addr(&bar));
        const bool done = tc::mbar_wait(tc::smem_addr(&bar), 0u, kMmaWait);
        ok[blockIdx.x] = done ? 1 : 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace
}  // namespace enufft

using namespace enufft;

extern "C" enufft_status enufft_probe_peaks(enufft_peaks* out, void* cuda_stream) {
    if (!out) {
        set_thread_error("probe_peaks: NULL output");
        return ENUFFT_ERR_ARG;
    }
    memset(out, 0, sizeof(*out));
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms < 1) {
        set_thread_error("probe_peaks: no device");
        return ENUFFT_ERR_CUDA;
    }
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    float* sink = nullptr;
    int* ok = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(float) * kProbeThreads)) != cudaSuccess ||
        (e = cudaMalloc(&ok, sizeof(int) * sms)) != cudaSuccess) {
        cudaFree(sink);
        set_thread_error("probe_peaks: cudaMalloc failed");
        return ENUFFT_ERR_NOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto launch) -> double {   // best of three after one warm-up, ms
        double best = 1e30;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            launch();
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        return best;
    };
    const int grid = 2 * sms;
    const double fma_ms = timed([&] { probe_fma_kernel<<<grid, kProbeThreads, 0, s>>>(sink, 1.0f); });
    out->fp32_tflops = 2.0 * grid * kProbeThreads * (double)kFmaIters * 8 / (fma_ms * 1e-3) / 1e12;
    const double nred = (double)grid * kProbeThreads * kRedIters * 8;
    const double r0 = timed([&] { probe_red_kernel<0><<<grid, kProbeThreads, 0, s>>>(sink); });
    const double r1 = timed([&] { probe_red_kernel<1><<<grid, kProbeThreads, 0, s>>>(sink); });
    const double r2 = timed([&] { probe_red_kernel<2><<<grid, kProbeThreads, 0, s>>>(sink); });
    out->smem_red_u32_gops = nred / (r0 * 1e-3) / 1e9;
    out->smem_red_u32_random_gops = nred / (r1 * 1e-3) / 1e9;
    out->smem_red_f32_gops = nred / (r2 * 1e-3) / 1e9;
    e = cudaFuncSetAttribute(probe_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaPadSmem);
    const double mma_ms = timed([&] { probe_mma_kernel<<<sms, 128, kMmaPadSmem, s>>>(ok); });
    int* hok = new int[sms];
    cudaMemcpy(hok, ok, sizeof(int) * sms, cudaMemcpyDeviceToHost);
    int good = 0;
    for (int i = 0; i < sms; ++i) good += hok[i];
    delete[] hok;
    out->f16_tflops = good == sms ? 2.0 * 128 * 256 * 16 * (double)kMmaIters * sms / (mma_ms * 1e-3) / 1e12 : 0.0;
    out->num_sms = sms;
    e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(ok);
    if (e != cudaSuccess) {
        set_thread_error(std::string("probe_peaks: ") + cudaGetErrorString(e));
        return ENUFFT_ERR_CUDA;
    }
    if (good != sms) {
        set_thread_error("probe_peaks: a tensor-core probe block's bounded wait expired");
        return ENUFFT_ERR_TIMEOUT;
    }
    return ENUFFT_OK;
}
