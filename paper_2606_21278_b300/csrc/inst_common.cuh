// inst_common.cuh -- instantiation helpers for the fused kernels (one translation unit per
// precision and grid size, so they compile in parallel).
#pragma once

#include "internal.h"

namespace enufft {

template <typename T, int NF, int W>
cudaError_t prepare_impl(int* fwd_per_sm, int* adj_per_sm) {
    using CF = FwdCfg<T, NF, W>;
    cudaError_t e = cudaFuncSetAttribute(type1_fused_kernel<T, NF, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CF::smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(type1_adjoint_kernel<T, NF, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CF::smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fwd_per_sm, type1_fused_kernel<T, NF, W>, CF::NT,
                                                      CF::smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(adj_per_sm, type1_adjoint_kernel<T, NF, W>, CF::NT,
                                                         CF::smem_bytes);
}

template <typename T, int NF, int W>
cudaError_t launch_fwd_impl(const FwdArgs<T>& a, int grid, cudaStream_t s) {
    using CF = FwdCfg<T, NF, W>;
    type1_fused_kernel<T, NF, W><<<grid, CF::NT, CF::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int NF, int W>
cudaError_t launch_adj_impl(const AdjArgs<T>& a, int grid, cudaStream_t s) {
    using CF = FwdCfg<T, NF, W>;
    type1_adjoint_kernel<T, NF, W><<<grid, CF::NT, CF::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace enufft

// Defines the per-translation-unit entry points for precision T and grid size NF over the
// kernel widths listed in WIDTHS(X).
#define ENUFFT_DEFINE_UNIT(SUFFIX, T, NF, WIDTHS)                                                   \
    namespace enufft {                                                                             \
    cudaError_t prepare_##SUFFIX(int w, int* f, int* a) {                                          \
        switch (w) {                                                                               \
            WIDTHS(ENUFFT_PREP_CASE_##SUFFIX)                                                      \
        }                                                                                          \
        return cudaErrorInvalidValue;                                                              \
    }                                                                                              \
    cudaError_t launch_fwd_##SUFFIX(const FwdArgs<T>& args, int w, int grid, cudaStream_t s) {     \
        switch (w) {                                                                               \
            WIDTHS(ENUFFT_FWD_CASE_##SUFFIX)                                                       \
        }                                                                                          \
        return cudaErrorInvalidValue;                                                              \
    }                                                                                              \
    cudaError_t launch_adj_##SUFFIX(const AdjArgs<T>& args, int w, int grid, cudaStream_t s) {     \
        switch (w) {                                                                               \
            WIDTHS(ENUFFT_ADJ_CASE_##SUFFIX)                                                       \
        }                                                                                          \
        return cudaErrorInvalidValue;                                                              \
    }                                                                                              \
    size_t smem_##SUFFIX(int w) {                                                                  \
        switch (w) {                                                                               \
            WIDTHS(ENUFFT_SMEM_CASE_##SUFFIX)                                                      \
        }                                                                                          \
        return 0;                                                                                  \
    }                                                                                              \
    }
