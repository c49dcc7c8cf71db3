// internal.h -- launch interface between the C-ABI host code and the kernel instantiations.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "enufft.h"
#include "adjoint.cuh"
#include "forward.cuh"

namespace enufft {

// Edge-aligned frame (App. A, Eq. rotation_matrix): each cell's centroid and rotation, kept beside
// its CellConst, whose frame is then the local one (origin 0, rotated vertices).
struct FrameRot {
    double cx, cy;   // centroid x-bar
    double c, s;     // R = [[c, s], [-s, c]]
};
// Per-call pre-pass of edge-frame plans (edge_frame.cu): the local coordinates v = R (x - x-bar) of
// every sample into (vx, vy), see enufft_frame.
cudaError_t launch_edge_frame(bool dbl, const void* x, const void* y, const int64_t* offsets, const CellConst* cells,
                              const FrameRot* rot, int64_t n_cells, void* vx, void* vy, unsigned* status, int grid,
                              cudaStream_t s);

// Is (precision, n_f, W) compiled?  Shared-memory bytes and threads of the fused kernels.
bool fused_supported(bool dbl, int nf, int w);
size_t fused_smem_bytes(bool dbl, int nf, int w);
int fused_threads(int nf);
// Raise the dynamic shared-memory limit of both kernels of (precision, n_f, W) and return the
// number of co-resident blocks per SM of the forward (fwd) and adjoint (adj) kernels.
cudaError_t fused_prepare(bool dbl, int nf, int w, int* fwd_per_sm, int* adj_per_sm);

cudaError_t launch_type1(const FwdArgs<float>& a, int nf, int w, int grid, cudaStream_t s);
cudaError_t launch_type1(const FwdArgs<double>& a, int nf, int w, int grid, cudaStream_t s);
cudaError_t launch_adjoint(const AdjArgs<float>& a, int nf, int w, int grid, cudaStream_t s);
cudaError_t launch_adjoint(const AdjArgs<double>& a, int nf, int w, int grid, cudaStream_t s);

// Large-grid (n_f = 256) pipeline, see large.cuh.
struct LargeArgs;
struct LargeFftArgs;
cudaError_t large_prepare(int P);
cudaError_t large_run_batch(const LargeArgs& la, int nbin_blocks, int nwork, const LargeFftArgs& fa, int W, int lt,
                            int fft_grid, cudaStream_t s);
struct LargeAdjFftArgs;
struct LargeInterpArgs;
// adjoint (mode 0) or reconstruction (mode 1) of one batch: per-cell inverse transforms into the
// batch's fine grids, interpolation per work item, and (mode 1) the per-cell diagnostics
cudaError_t large_run_adjoint_batch(const LargeAdjFftArgs& fa, const LargeInterpArgs& ia, int nwork, int W,
                                    int fft_grid, double* stats, const CellConst* cells, cudaStream_t s);

// Plain binary32 per-cell path (plain.cu): one launch sequence per cell.
struct PlainRun {
    const float *x, *y, *h, *w;
    const int64_t* h_off;          // host copy of the CSR offsets
    int64_t n_cells;
    const CellConst* cells;
    int NF, W, P;
    float beta;                    // kernel shape (ES beta or KB gamma)
    int kind;                      // KERNEL_ES or KERNEL_KB
    float inv_norm;                // KB: 1 / I0(gamma)
    const double* inv_phi;         // host, P/2 + 1 entries
    const cplx<float>* twiddle;    // device, W_NF^j
    float* grid;                   // device scratch, NF * NF
    cplx<float>* buf;              // device scratch, NF * NF
    cplx<float>* coeffs;
    unsigned* status;
};
cudaError_t plain_run(const PlainRun& r, cudaStream_t s);

// Tensor-core direct NUDFT of small cells (tc_nudft.cu), P <= 64, binary32 samples.
struct TcLaunch {
    const float *x, *y, *h, *w;
    const int64_t* offsets;
    const CellConst* cells;
    const int* list;               // device, cells routed here
    int n_list, P, NF, num_sms;
    cplx<float>* coeffs;
    unsigned* status;
    const EmsArgs* ems;            // NULL: no EMS ranking
    EmsScratch ems_out;
};
cudaError_t tc_prepare();
cudaError_t launch_wait_timeout(unsigned polls, unsigned* status, cudaStream_t s);
cudaError_t launch_tc_nudft(const TcLaunch& l, cudaStream_t s);

// Voronoi quadrature weights by raster sampling (voronoi.cu), binary32 samples.
cudaError_t launch_voronoi(const float* x, const float* y, const int64_t* offsets, const CellConst* cells, int n_cells,
                           int Ng, float* w, unsigned* status, int num_sms, cudaStream_t s);

// Plan-time route tuning (autotune.cu).
struct TuneEnv {
    const CellConst* cells;   // the plan's cells (device)
    int n_cells;
    int P, NF, W;
    KernelPoly poly;
    double beta;
    const double* inv_phi;    // host, P/2 + 1 entries
    const void* twiddle;      // device
    int num_sms, fwd_per_sm;  // SMs; resident fused blocks per SM
    unsigned* status;
    cudaStream_t stream;
    int tc_cap;               // largest cell size the caller allows on the tensor cores (0: none)
    int q_median;             // the plan's median cell size
};
cudaError_t autotune_run(const TuneEnv& env, enufft_tuning* out);
// synthetic samples of ncells cells (counts from offsets, written at offset - p0), uniform over each
// cell's window: the tile tuning of the large route
cudaError_t large_tune_samples(const CellConst* cells, const int64_t* offsets, int64_t p0, int ncells, float* x,
                               float* y, float* h, float* w, cudaStream_t s);
bool tune_cache_get(const char* path, const std::string& key, enufft_tuning* out);
bool tune_cache_put(const char* path, const std::string& key, const enufft_tuning& t);

// Record the calling thread's last error text (read back by enufft_last_error(NULL)).
void set_thread_error(const std::string& msg);

}  // namespace enufft
