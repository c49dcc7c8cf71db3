// inst_f32_64.cu -- fused forward/adjoint kernels, float, n_f = 64.
#include "inst_common.cuh"

#define WIDTHS_f32_64(X) X(4) X(5) X(6) X(7) X(8) X(9) X(10)
#define ENUFFT_PREP_CASE_f32_64(W) case W: return prepare_impl<float, 64, W>(f, a);
#define ENUFFT_FWD_CASE_f32_64(W) case W: return launch_fwd_impl<float, 64, W>(args, grid, s);
#define ENUFFT_ADJ_CASE_f32_64(W) case W: return launch_adj_impl<float, 64, W>(args, grid, s);
#define ENUFFT_SMEM_CASE_f32_64(W) case W: return FwdCfg<float, 64, W>::smem_bytes;

ENUFFT_DEFINE_UNIT(f32_64, float, 64, WIDTHS_f32_64)
