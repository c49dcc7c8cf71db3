// noalloc.cu -- Elastic Mode Selection of binary32 spectra with no device allocation.
//
// Some callers cannot allocate device memory at the moment they need EMS: code running where a
// cudaMalloc would implicitly synchronise the device and stall other streams of a latency-bound
// pipeline, processes whose device memory is owned by another allocator (a framework's memory
// pool), or plug-ins that are not allowed to own device memory at all.  This entry point serves
// them: it needs no plan and calls no allocating routine.  Its per-cell scratch (the ranked keys
// between the two EMS stages) lives in one fixed file-scope device array of
// kNoAllocMaxCells cells, which every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "enufft.h"
#include "internal.h"
#include "kernels_misc.cuh"

using namespace enufft;

namespace {

constexpr int64_t kNoAllocMaxCells = 2048;
constexpr size_t kKeyBytes = sizeof(EmsKey) * (size_t)kEmsMaxK * kNoAllocMaxCells;
constexpr size_t kInfoBytes = sizeof(EmsCellInfo) * (size_t)kNoAllocMaxCells;

// the shared scratch (about 2.2 MB): ranked keys, then per-cell counts
static __device__ __align__(256) unsigned char g_noalloc_scratch[kKeyBytes + kInfoBytes];

// device address of g_noalloc_scratch per device; host code must not use the symbol itself
constexpr int kMaxDevices = 128;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

enufft_status fail(enufft_status st, const char* msg) {
    set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" enufft_status enufft_ems_noalloc(int modes, int64_t n_cells, const void* d_coeffs,
                                            const double* d_mode_weights, int mode_weights_per_cell,
                                            const enufft_ems_params* prm, int32_t* d_kstar, int32_t* d_sel,
                                            double* d_retained_power, void* cuda_stream) {
    if (!prm) return fail(ENUFFT_ERR_ARG, "ems_noalloc: params is NULL");
    if (prm->k_max < 1 || prm->k_max > kEmsMaxK) return fail(ENUFFT_ERR_ARG, "ems_noalloc: k_max must be in [1, 64]");
    if (prm->k_min < 0 || prm->k_min > prm->k_max) return fail(ENUFFT_ERR_ARG, "ems_noalloc: k_min must be in [0, k_max]");
    if (!(prm->delta > 0.0)) return fail(ENUFFT_ERR_ARG, "ems_noalloc: delta must be positive");
    if (modes < 2 || modes > 2 * kMaxHalf || (modes & 1))
        return fail(ENUFFT_ERR_ARG, "ems_noalloc: modes must be even and in [2, 128]");
    if (n_cells < 0) return fail(ENUFFT_ERR_ARG, "ems_noalloc: n_cells < 0");
    if (n_cells > kNoAllocMaxCells)
        return fail(ENUFFT_ERR_ARG, "ems_noalloc: n_cells exceeds the fixed scratch of 2048 cells; "
                                    "split the batch or use enufft_ems with a plan");
    if (n_cells == 0) return ENUFFT_OK;
    if (!d_coeffs || !d_kstar || !d_sel || !d_retained_power)
        return fail(ENUFFT_ERR_ARG, "ems_noalloc: NULL data pointer");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(ENUFFT_ERR_CUDA, "ems_noalloc: cudaGetDevice failed");
    void* base = nullptr;
    {   // once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
            if (e != cudaSuccess) return fail(ENUFFT_ERR_CUDA, "ems_noalloc: cudaGetSymbolAddress failed");
            g_scratch_addr[dev] = base;
        }
        base = g_scratch_addr[dev];
    }
    EmsScratch sc;
    sc.keys = reinterpret_cast<EmsKey*>(base);
    sc.info = reinterpret_cast<EmsCellInfo*>(reinterpret_cast<unsigned char*>(base) + kKeyBytes);

    EmsArgs ea;
    ea.k_min = prm->k_min;
    ea.k_max = prm->k_max;
    ea.alpha_min = prm->alpha_min;
    ea.alpha_max = prm->alpha_max;
    ea.delta = prm->delta;
    ea.w1 = prm->w1;
    ea.w2 = prm->w2;
    ea.sum_over = prm->sum_over ? 1 : 0;
    ea.include_dc = prm->include_dc ? 1 : 0;
    ea.W = d_mode_weights;
    ea.w_per_cell = mode_weights_per_cell ? 1 : 0;
    ea.kstar = d_kstar;
    ea.sel = d_sel;
    ea.retained = d_retained_power;

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    const int grid = (int)(n_cells < (int64_t)sms * 4 ? n_cells : (int64_t)sms * 4);
    const size_t smem = ems_smem_bytes(16, prm->k_max);
    const int half = modes / 2, lim = half - 1;
    const int J = (lim > 0 ? lim * (2 * lim + 2) : 0) + 1;
    if (J > 512 * 4)
        ems_rank_kernel<float, 16><<<grid, 512, smem, s>>>((const cplx<float>*)d_coeffs, modes, n_cells, ea, sc);
    else
        ems_rank_kernel<float, 4><<<grid, 512, smem, s>>>((const cplx<float>*)d_coeffs, modes, n_cells, ea, sc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ENUFFT_ERR_CUDA, "ems_noalloc: ranking launch failed");
    ems_finish_kernel<<<(unsigned)((n_cells + 127) / 128), 128, 0, s>>>(n_cells, ea, sc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ENUFFT_ERR_CUDA, "ems_noalloc: finish launch failed");
    return ENUFFT_OK;
}
