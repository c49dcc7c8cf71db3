// inst_f32_128.cu -- fused forward/adjoint kernels, float, n_f = 128.
#include "inst_common.cuh"

#define WIDTHS_f32_128(X) X(4) X(5) X(6) X(7) X(8) X(9) X(10)
#define ENUFFT_PREP_CASE_f32_128(W) case W: return prepare_impl<float, 128, W>(f, a);
#define ENUFFT_FWD_CASE_f32_128(W) case W: return launch_fwd_impl<float, 128, W>(args, grid, s);
#define ENUFFT_ADJ_CASE_f32_128(W) case W: return launch_adj_impl<float, 128, W>(args, grid, s);
#define ENUFFT_SMEM_CASE_f32_128(W) case W: return FwdCfg<float, 128, W>::smem_bytes;

ENUFFT_DEFINE_UNIT(f32_128, float, 128, WIDTHS_f32_128)
