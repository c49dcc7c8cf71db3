// inst_f64_128.cu -- fused forward/adjoint kernels, double, n_f = 128.
#include "inst_common.cuh"

#define WIDTHS_f64_128(X) X(8) X(9) X(10)
#define ENUFFT_PREP_CASE_f64_128(W) case W: return prepare_impl<double, 128, W>(f, a);
#define ENUFFT_FWD_CASE_f64_128(W) case W: return launch_fwd_impl<double, 128, W>(args, grid, s);
#define ENUFFT_ADJ_CASE_f64_128(W) case W: return launch_adj_impl<double, 128, W>(args, grid, s);
#define ENUFFT_SMEM_CASE_f64_128(W) case W: return FwdCfg<double, 128, W>::smem_bytes;

ENUFFT_DEFINE_UNIT(f64_128, double, 128, WIDTHS_f64_128)
