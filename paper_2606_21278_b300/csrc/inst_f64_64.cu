// inst_f64_64.cu -- fused forward/adjoint kernels, double, n_f = 64.
#include "inst_common.cuh"

#define WIDTHS_f64_64(X) X(8) X(9) X(10) X(11) X(12) X(13)
#define ENUFFT_PREP_CASE_f64_64(W) case W: return prepare_impl<double, 64, W>(f, a);
#define ENUFFT_FWD_CASE_f64_64(W) case W: return launch_fwd_impl<double, 64, W>(args, grid, s);
#define ENUFFT_ADJ_CASE_f64_64(W) case W: return launch_adj_impl<double, 64, W>(args, grid, s);
#define ENUFFT_SMEM_CASE_f64_64(W) case W: return FwdCfg<double, 64, W>::smem_bytes;

ENUFFT_DEFINE_UNIT(f64_64, double, 64, WIDTHS_f64_64)
