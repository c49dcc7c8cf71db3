// api.cu -- host side of the C ABI declared in include/enufft.h.
//
// Plan creation does the per-plan constant work once: kernel width and shape (ES kernel,
// exponential of semicircle), its piecewise polynomial for binary32 evaluation, the kernel's
// Fourier transform Phi(k) for the deconvolution (Gauss-Legendre quadrature, binary64), the FFT
// twiddles, the per-cell frames (device kernel, binary64) and the size-ordered work lists.
// Execution calls only marshal arguments and launch kernels on the plan's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "enufft.h"
#include "internal.h"
#include "kernels_misc.cuh"
#include "large_args.cuh"
#include "large_adj.cuh"

using namespace enufft;

namespace enufft {
cudaError_t prepare_f32_64(int, int*, int*);
cudaError_t prepare_f32_128(int, int*, int*);
cudaError_t prepare_f64_64(int, int*, int*);
cudaError_t prepare_f64_128(int, int*, int*);
cudaError_t launch_fwd_f32_64(const FwdArgs<float>&, int, int, cudaStream_t);
cudaError_t launch_fwd_f32_128(const FwdArgs<float>&, int, int, cudaStream_t);
cudaError_t launch_fwd_f64_64(const FwdArgs<double>&, int, int, cudaStream_t);
cudaError_t launch_fwd_f64_128(const FwdArgs<double>&, int, int, cudaStream_t);
cudaError_t launch_adj_f32_64(const AdjArgs<float>&, int, int, cudaStream_t);
cudaError_t launch_adj_f32_128(const AdjArgs<float>&, int, int, cudaStream_t);
cudaError_t launch_adj_f64_64(const AdjArgs<double>&, int, int, cudaStream_t);
cudaError_t launch_adj_f64_128(const AdjArgs<double>&, int, int, cudaStream_t);
size_t smem_f32_64(int);
size_t smem_f32_128(int);
size_t smem_f64_64(int);
size_t smem_f64_128(int);

size_t fused_smem_bytes(bool dbl, int nf, int w) {
    if (dbl) return nf == 64 ? smem_f64_64(w) : nf == 128 ? smem_f64_128(w) : 0;
    return nf == 64 ? smem_f32_64(w) : nf == 128 ? smem_f32_128(w) : 0;
}
bool fused_supported(bool dbl, int nf, int w) {
    const size_t b = fused_smem_bytes(dbl, nf, w);
    return b > 0 && b <= 232448;
}
int fused_threads(int nf) { return nf >= 128 ? 512 : 256; }
cudaError_t fused_prepare(bool dbl, int nf, int w, int* f, int* a) {
    if (dbl) return nf == 64 ? prepare_f64_64(w, f, a) : prepare_f64_128(w, f, a);
    return nf == 64 ? prepare_f32_64(w, f, a) : prepare_f32_128(w, f, a);
}
cudaError_t launch_type1(const FwdArgs<float>& a, int nf, int w, int grid, cudaStream_t s) {
    return nf == 64 ? launch_fwd_f32_64(a, w, grid, s) : launch_fwd_f32_128(a, w, grid, s);
}
cudaError_t launch_type1(const FwdArgs<double>& a, int nf, int w, int grid, cudaStream_t s) {
    return nf == 64 ? launch_fwd_f64_64(a, w, grid, s) : launch_fwd_f64_128(a, w, grid, s);
}
cudaError_t launch_adjoint(const AdjArgs<float>& a, int nf, int w, int grid, cudaStream_t s) {
    return nf == 64 ? launch_adj_f32_64(a, w, grid, s) : launch_adj_f32_128(a, w, grid, s);
}
cudaError_t launch_adjoint(const AdjArgs<double>& a, int nf, int w, int grid, cudaStream_t s) {
    return nf == 64 ? launch_adj_f64_64(a, w, grid, s) : launch_adj_f64_128(a, w, grid, s);
}
}  // namespace enufft

// ------------------------------------------------------------------------------------------------
// plan
// ------------------------------------------------------------------------------------------------
struct enufft_plan_s {
    enufft_opts opts;
    int P = 0, NF = 0, W = 0;
    double beta = 0.0, sigma_eff = 0.0, poly_err = 0.0;
    bool dbl = false;
    int64_t n_cells = 0, n_points = 0;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    CellConst* d_cells = nullptr;
    int64_t* d_offsets = nullptr;
    int* d_order = nullptr;          // all cells, largest first
    int n_fused = 0;
    int n_tc = 0;                    // cells d_order[n_fused ..) take the tensor-core direct sum
    unsigned* d_ctr = nullptr;       // [0] forward ticket, [1] adjoint ticket, [2] status
    EmsScratch ems_scratch = {nullptr, nullptr};   // stage-1 EMS results per cell
    void* d_twiddle = nullptr;
    int fwd_per_sm = 0, adj_per_sm = 0;
    int fwd_grid_per_sm = 0;         // persistent fused blocks launched per SM (tuned or fwd_per_sm)
    int tc_threshold = 0;            // routing threshold in effect
    bool tuned = false;
    enufft_tuning tuning = {};
    double inv_phi[kMaxHalf + 1] = {};
    KernelPoly poly = {};
    // large-grid (n_f = 256) route: cells in batches with bounded scratch
    bool large = false;
    struct LBatch {
        int cell0, ncells, block0, nblocks, work0, nwork;
        int64_t p0;
    };
    std::vector<LBatch> lbatches;
    int4* d_lblocks = nullptr;
    int2* d_lcellblk = nullptr;      // per cell: {first sort block relative to its batch, count}
    int4* d_lwork = nullptr;         // spread work items of all batches (per batch: largest cells first)
    int* d_lblk_off = nullptr;       // [sort blocks of a batch][65] tile offsets
    float* d_lblk_abs = nullptr;     // [sort blocks of a batch][64] per-tile |c| sums
    float4* d_lrec = nullptr;
    unsigned long long* d_lgrid = nullptr;   // fixed-point fine grids of one batch
    int* d_lexp = nullptr;                   // their scales
    double* d_lpartial = nullptr;            // reconstruction: per work item partial sums [max items][3]
    double* d_lspec = nullptr;               // reconstruction: per cell spectral variances [n_cells][2]
    int lmax_cells = 0;
    int lt = kLT;                            // tile side of the sorted spreading (16, 32 or 64)
    // edge-aligned frame: per-cell centroid and rotation, per-call local coordinates of the samples
    bool edge = false;
    FrameRot* d_rot = nullptr;
    void* d_vx = nullptr;
    void* d_vy = nullptr;
    // plain binary32 per-cell path
    bool plain = false;
    std::vector<int64_t> h_off;
    float* d_pgrid = nullptr;
    void* d_pbuf = nullptr;
    // plan-owned CUDA graph of enufft_type1_ems and the arguments it was captured with
    struct GraphKey {
        const void *x, *y, *h, *w;
        void* coeffs;
        const double* mw;
        int per_cell;
        enufft_ems_params prm;
        int32_t *kstar, *sel;
        double* ret;
    };
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    GraphKey gkey = {};
    std::string err;
};

static enufft_status tune_large_tile(enufft_plan p, const std::vector<int64_t>& off, enufft_tuning* t);

// key of a plan configuration in the tuning cache: the configuration on this kind of GPU
static std::string tune_key(enufft_plan p, const enufft_opts& o, int NF, int W) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, p->device);
    std::string gpu = prop.name;
    for (char& c : gpu)
        if (c == '"' || c == '\\') c = '_';
    char key[384];
    snprintf(key, sizeof key, "gpu=%s|sms=%d|P=%d|nf=%d|w=%d|prec=%d|kernel=%d|frame=%d|tc_cap=%d", gpu.c_str(),
             p->num_sms, p->P, NF, W, (int)o.prec, (int)o.kernel, (int)o.frame, o.tc_max_points);
    return key;
}

// batch bounds of the large route: records (16 B per sample) and fine grids (256 KB per cell)
static constexpr int64_t kLargeBatchPoints = (int64_t)1 << 26;
static constexpr int kLargeBatchCells = 512;

static thread_local std::string g_last_error;

void enufft::set_thread_error(const std::string& msg) { g_last_error = msg; }

static enufft_status fail(enufft_plan p, enufft_status st, const std::string& msg) {
    if (p)
        p->err = msg;
    else
        g_last_error = msg;
    return st;
}
static enufft_status cuda_fail(enufft_plan p, cudaError_t e, const char* where) {
    return fail(p, e == cudaErrorMemoryAllocation ? ENUFFT_ERR_NOMEM : ENUFFT_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

// the spreading kernel on z in [-1, 1] (z = 2 tau / W, tau in grid points), host side in binary64:
// ES exp(beta (sqrt(1 - z^2) - 1)), or KB I0(gamma sqrt(1 - z^2)) / I0(gamma) (Eq. kb_compact
// normalised to 1 at the centre)
struct HostKernel {
    int kind;
    double shape;      // ES beta or KB gamma
    double inv_norm;   // KB: 1 / I0(gamma)
    double operator()(double z) const {
        if (std::fabs(z) > 1.0) return 0.0;
        const double r = std::sqrt(1.0 - z * z);
        return kind == ENUFFT_KERNEL_KB ? std::cyl_bessel_i(0.0, shape * r) * inv_norm : std::exp(shape * (r - 1.0));
    }
};

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the Legendre recurrence)
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wts) {
    x.resize(n);
    wts.resize(n);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        wts[i] = wts[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Phi(k) = integral of phi(2 tau / W) e^{-2 pi i k tau / nf} d tau (grid units), the kernel's
// Fourier transform used by the deconvolution (Sec. 2.1.2, Eq. deconv).  ES: Gauss-Legendre
// quadrature.  KB: Eq. kb_fourier with a = W/2 and a k-independent factor 1/I0(gamma) in place of
// 1/I0(beta) (the normalisation of the kernel): 2a sinh(s)/s, s = sqrt(gamma^2 - (a omega)^2),
// omega = 2 pi k / nf, continued as 2a sin(s')/s', s' = sqrt((a omega)^2 - gamma^2), beyond gamma.
static double kernel_ft(int k, int W, int nf, const HostKernel& ker, const std::vector<double>& x,
                        const std::vector<double>& wts) {
    const double pi = 3.14159265358979323846;
    if (ker.kind == ENUFFT_KERNEL_KB) {
        const double a = 0.5 * W, ao = a * 2.0 * pi * k / nf;
        const double d = ker.shape * ker.shape - ao * ao;
        double f;
        if (d > 0.0) {
            const double r = std::sqrt(d);
            f = std::sinh(r) / r;
        } else if (d < 0.0) {
            const double r = std::sqrt(-d);
            f = std::sin(r) / r;
        } else {
            f = 1.0;
        }
        return 2.0 * a * f * ker.inv_norm;
    }
    double s = 0.0;
    for (size_t i = 0; i < x.size(); ++i) s += wts[i] * ker(x[i]) * std::cos(pi * k * W * x[i] / nf);
    return 0.5 * W * s;
}

// Piece i of the kernel as a function of t in [0, 1): phi((t - W/2 + i) 2 / W); fit on
// u = 2t - 1 by Chebyshev interpolation with `deg` coefficients, returned as monomials in u.
static double fit_pieces(int W, const HostKernel& ker, int deg, KernelPoly& kp) {
    const double pi = 3.14159265358979323846;
    kp.w = W;
    kp.deg = deg;
    kp.beta = (float)ker.shape;
    kp.kind = ker.kind;
    kp.inv_norm = ker.inv_norm;
    for (int i = 0; i < kMaxW; ++i)
        for (int d = 0; d < kMaxDeg; ++d) kp.c[i][d] = 0.0f;
    double maxerr = 0.0;
    for (int i = 0; i < W; ++i) {
        auto f = [&](double u) { return ker(((u + 1.0) * 0.5 - 0.5 * W + i) * 2.0 / W); };
        std::vector<double> a(deg, 0.0), fk(deg);
        for (int k = 0; k < deg; ++k) fk[k] = f(std::cos(pi * (k + 0.5) / deg));
        for (int j = 0; j < deg; ++j) {
            double s = 0.0;
            for (int k = 0; k < deg; ++k) s += fk[k] * std::cos(pi * j * (k + 0.5) / deg);
            a[j] = (j == 0 ? 1.0 : 2.0) * s / deg;
        }
        // Chebyshev -> monomial: T_0 = 1, T_1 = u, T_{j+1} = 2 u T_j - T_{j-1}
        std::vector<double> mono(deg, 0.0), tm1(deg, 0.0), t0(deg, 0.0), t1(deg, 0.0);
        t0[0] = 1.0;
        for (int j = 0; j < deg; ++j) {
            const std::vector<double>& tj = (j == 0) ? t0 : t1;
            for (int d = 0; d < deg; ++d) mono[d] += a[j] * tj[d];
            std::vector<double> nx(deg, 0.0);
            if (j == 0) {
                if (deg > 1) nx[1] = 1.0;
                tm1 = t0;
                t1 = nx;
            } else {
                for (int d = 0; d + 1 < deg; ++d) nx[d + 1] += 2.0 * t1[d];
                for (int d = 0; d < deg; ++d) nx[d] -= tm1[d];
                tm1 = t1;
                t1 = nx;
            }
        }
        for (int d = 0; d < deg; ++d) kp.c[i][d] = (float)mono[d];
        for (int s = 0; s <= 400; ++s) {
            const double u = -1.0 + 2.0 * s / 400.0;
            double v = 0.0;
            for (int d = deg - 1; d >= 0; --d) v = v * u + mono[d];
            maxerr = std::max(maxerr, std::fabs(v - f(u)));
        }
    }
    return maxerr;
}

extern "C" {

void enufft_default_opts(enufft_opts* o) {
    if (!o) return;
    o->modes = 64;
    o->oversamp = 2.0;
    o->kernel_width = 7;
    o->tol = 0.0;
    o->prec = ENUFFT_MIXED;
    o->mask = ENUFFT_MASK_CELL;
    o->eta = 1.5;
    o->tc_max_points = 0;
    o->kernel = ENUFFT_KERNEL_ES;
    o->frame = ENUFFT_FRAME_CENTROID;
    o->autotune = 0;
    o->tune_cache = nullptr;
    o->deterministic = 1;
}

void enufft_default_ems(enufft_ems_params* p) {
    if (!p) return;
    p->k_min = 1;
    p->k_max = 12;
    p->alpha_min = 0.0;
    p->alpha_max = 0.7;
    p->delta = 0.02;
    p->w1 = 0.5;
    p->w2 = 0.5;
    p->sum_over = 0;
    p->include_dc = 0;
}

const char* enufft_last_error(enufft_plan plan) { return plan ? plan->err.c_str() : g_last_error.c_str(); }

enufft_status enufft_plan_destroy(enufft_plan p) {
    if (!p) return ENUFFT_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaStreamSynchronize(p->stream);
    cudaFree(p->d_cells);
    cudaFree(p->d_offsets);
    cudaFree(p->d_order);
    cudaFree(p->d_ctr);
    cudaFree(p->d_twiddle);
    cudaFree(p->ems_scratch.keys);
    cudaFree(p->ems_scratch.info);
    cudaFree(p->d_lblocks);
    cudaFree(p->d_lcellblk);
    cudaFree(p->d_lwork);
    cudaFree(p->d_lblk_off);
    cudaFree(p->d_lblk_abs);
    cudaFree(p->d_lrec);
    cudaFree(p->d_lgrid);
    cudaFree(p->d_lexp);
    cudaFree(p->d_lpartial);
    cudaFree(p->d_lspec);
    cudaFree(p->d_pgrid);
    cudaFree(p->d_pbuf);
    cudaFree(p->d_rot);
    cudaFree(p->d_vx);
    cudaFree(p->d_vy);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->gstream) cudaStreamDestroy(p->gstream);
    cudaSetDevice(cur);
    delete p;
    return ENUFFT_OK;
}

enufft_status enufft_plan_create(enufft_plan* out, const enufft_opts* opts, int64_t n_cells,
                                 const int64_t* d_cell_offsets, const int32_t* d_cell_nverts,
                                 const double* d_cell_verts, void* cuda_stream) {
    if (!out) return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: out is NULL");
    *out = nullptr;
    if (!opts) return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: opts is NULL");
    if (n_cells < 0 || n_cells > (int64_t)0x7fffffff)
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: n_cells out of range");
    if (n_cells > 0 && (!d_cell_offsets || !d_cell_nverts || !d_cell_verts))
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: NULL cell array");
    const enufft_opts& o = *opts;
    if (o.modes < 2 || o.modes > 2 * kMaxHalf || (o.modes & 1))
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: modes must be even and in [2, 128]");
    if (!(o.oversamp >= 2.0) || o.oversamp > 16.0)
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: oversamp must be in [2, 16]");
    if (o.kernel_width < 2 || o.kernel_width > kMaxW)
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: kernel_width must be in [2, 16]");
    if (o.prec != ENUFFT_FP64 && o.prec != ENUFFT_FP32 && o.prec != ENUFFT_MIXED)
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: bad precision");
    if (o.mask < 0 || o.mask > 2) return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: bad mask");
    if (!(o.eta > 0.0)) return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: eta must be positive");
    if (o.tol < 0.0 || o.tol >= 1.0) return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: tol must be in [0, 1)");
    if (o.tc_max_points < 0) return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: tc_max_points < 0");
    if (o.kernel != ENUFFT_KERNEL_ES && o.kernel != ENUFFT_KERNEL_KB)
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: bad kernel");
    if (o.frame != ENUFFT_FRAME_CENTROID && o.frame != ENUFFT_FRAME_EDGE)
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: bad frame");
    if (o.autotune != 0 && o.autotune != 1) return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: autotune must be 0 or 1");
    if (o.deterministic != 0 && o.deterministic != 1)
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: deterministic must be 0 or 1");

    enufft_plan p = new enufft_plan_s();
    p->opts = o;
    p->P = o.modes;
    p->dbl = o.prec == ENUFFT_FP64;
    p->n_cells = n_cells;
    p->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        enufft_status st = cuda_fail(nullptr, e, "cudaGetDevice");
        delete p;
        return st;
    }
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);

    // kernel width from the tolerance (ES kernel at sigma = 2: about one digit per grid point)
    int W = o.kernel_width;
    if (o.tol > 0.0) W = std::max(W, (int)std::ceil(std::log10(1.0 / o.tol)) + 1);
    W = std::min(W, kMaxW);
    // fine grid: smallest power of two >= sigma * P, at least 64
    int NF = 64;
    while (NF < o.oversamp * o.modes) NF *= 2;
    p->W = W;
    p->NF = NF;
    p->sigma_eff = (double)NF / o.modes;
    HostKernel ker = {o.kernel, 0.0, 1.0};
    if (o.kernel == ENUFFT_KERNEL_KB) {
        // KB shape of Eq. kaisal_bessel_coeffs: beta = 2.34, gamma = pi sqrt((2 a beta / pi)^2 - 0.8),
        // half-width a = W / 2 grid points
        const double pi = 3.14159265358979323846, bkb = 2.34, t = W * bkb / pi;
        ker.shape = pi * std::sqrt(t * t - 0.8);
        ker.inv_norm = 1.0 / std::cyl_bessel_i(0.0, ker.shape);
    } else {
        // ES shape: beta = 2.30 W at sigma = 2, scaled by (1 - 1/(2 sigma)) for other sigma
        ker.shape = 2.30 * W * (1.0 - 0.5 / p->sigma_eff) / 0.75;
    }
    p->beta = ker.shape;
    p->plain = o.prec == ENUFFT_FP32;
    if (p->plain && NF > 256) {
        enufft_plan_destroy(p);
        return fail(nullptr, ENUFFT_ERR_UNSUPPORTED, "plan_create: the plain FP32 path supports n_f <= 256");
    }
    p->large = (NF == kLNF && !p->dbl && !p->plain);
    if (p->large && (W < 4 || W > 8 || o.modes > 2 * kMaxHalfL)) {
        enufft_plan_destroy(p);
        return fail(nullptr, ENUFFT_ERR_UNSUPPORTED, "plan_create: the n_f = 256 route supports widths 4..8");
    }
    if (!p->large && !p->plain && (NF > 128 || !fused_supported(p->dbl, NF, W))) {
        enufft_plan_destroy(p);
        char buf[160];
        snprintf(buf, sizeof buf, "plan_create: no kernel for %s n_f=%d width=%d", p->dbl ? "fp64" : "fp32", NF, W);
        return fail(nullptr, ENUFFT_ERR_UNSUPPORTED, buf);
    }
    if (!p->dbl) {
        p->poly_err = fit_pieces(W, ker, poly_deg(W), p->poly);
    } else {
        p->poly.w = W;
        p->poly.beta = (float)p->beta;
        p->poly.kind = ker.kind;
        p->poly.inv_norm = ker.inv_norm;
    }
    {
        std::vector<double> gx, gw;
        gauss_legendre(256, gx, gw);
        for (int k = 0; k <= p->P / 2; ++k) p->inv_phi[k] = 1.0 / kernel_ft(k, W, NF, ker, gx, gw);
    }

    // device state
    const size_t tw_bytes = (size_t)NF * (p->dbl ? 16 : 8);
    if ((e = cudaMalloc(&p->d_ctr, 4 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_twiddle, tw_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_cells, sizeof(CellConst) * std::max<int64_t>(n_cells, 1))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_offsets, sizeof(int64_t) * (n_cells + 1))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_order, sizeof(int) * std::max<int64_t>(n_cells, 1))) != cudaSuccess ||
        (e = cudaMalloc(&p->ems_scratch.keys, sizeof(EmsKey) * kEmsMaxK * std::max<int64_t>(n_cells, 1))) != cudaSuccess ||
        (e = cudaMalloc(&p->ems_scratch.info, sizeof(EmsCellInfo) * std::max<int64_t>(n_cells, 1))) != cudaSuccess) {
        enufft_status st = cuda_fail(nullptr, e, "plan_create: cudaMalloc");
        enufft_plan_destroy(p);
        return st;
    }
    {
        const double pi = 3.14159265358979323846;
        if (p->dbl) {
            std::vector<double> tw(2 * NF);
            for (int j = 0; j < NF; ++j) { tw[2 * j] = std::cos(2 * pi * j / NF); tw[2 * j + 1] = -std::sin(2 * pi * j / NF); }
            e = cudaMemcpyAsync(p->d_twiddle, tw.data(), tw_bytes, cudaMemcpyHostToDevice, p->stream);
        } else {
            std::vector<float> tw(2 * NF);
            for (int j = 0; j < NF; ++j) {
                tw[2 * j] = (float)std::cos(2 * pi * j / NF);
                tw[2 * j + 1] = (float)-std::sin(2 * pi * j / NF);
            }
            e = cudaMemcpyAsync(p->d_twiddle, tw.data(), tw_bytes, cudaMemcpyHostToDevice, p->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    }
    std::vector<int64_t> off(n_cells + 1, 0);
    if (e == cudaSuccess && n_cells > 0) {
        e = cudaMemcpyAsync(off.data(), d_cell_offsets, sizeof(int64_t) * (n_cells + 1), cudaMemcpyDeviceToHost,
                            p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_ctr, 0, 4 * sizeof(unsigned), p->stream);
    if (e != cudaSuccess) {
        enufft_status st = cuda_fail(nullptr, e, "plan_create: copy");
        enufft_plan_destroy(p);
        return st;
    }
    if (off[0] != 0) {
        enufft_plan_destroy(p);
        return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: offsets[0] must be 0");
    }
    for (int64_t j = 0; j < n_cells; ++j)
        if (off[j + 1] < off[j]) {
            enufft_plan_destroy(p);
            return fail(nullptr, ENUFFT_ERR_ARG, "plan_create: offsets must be non-decreasing");
        }
    p->n_points = off[n_cells];
    // largest cells first (longest-processing-time order for the ticket queue); stable
    std::vector<int> order(n_cells);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    p->n_fused = (int)n_cells;
    if (o.tc_max_points > 0) {
        if (p->dbl || p->plain || p->large || p->P > 64) {
            enufft_plan_destroy(p);
            return fail(nullptr, ENUFFT_ERR_UNSUPPORTED,
                        "plan_create: the tensor-core route needs a mixed-precision plan with modes <= 64");
        }
        for (int64_t j = 0; j < n_cells; ++j)
            if (off[j + 1] - off[j] <= o.tc_max_points) ++p->n_tc;
        p->n_fused = (int)(n_cells - p->n_tc);
        p->tc_threshold = o.tc_max_points;
    }
    if (n_cells > 0) {
        e = cudaMemcpyAsync(p->d_order, order.data(), sizeof(int) * n_cells, cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_offsets, off.data(), sizeof(int64_t) * (n_cells + 1), cudaMemcpyHostToDevice,
                                p->stream);
        p->edge = o.frame == ENUFFT_FRAME_EDGE;
        if (e == cudaSuccess && p->edge) {
            const size_t vb = (size_t)std::max<int64_t>(p->n_points, 1) * (p->dbl ? 8 : 4);
            e = cudaMalloc(&p->d_rot, sizeof(FrameRot) * n_cells);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->d_rot, 0, sizeof(FrameRot) * n_cells, p->stream);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_vx, vb);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_vy, vb);
        }
        if (e == cudaSuccess) {
            frame_kernel<<<(unsigned)((n_cells + 127) / 128), 128, 0, p->stream>>>(
                n_cells, d_cell_nverts, d_cell_verts, o.eta, (int)o.mask, NF, p->edge ? 1 : 0, p->d_cells, p->d_rot);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) {
            enufft_status st = cuda_fail(nullptr, e, "plan_create: frames");
            enufft_plan_destroy(p);
            return st;
        }
    } else {
        cudaMemsetAsync(p->d_offsets, 0, sizeof(int64_t), p->stream);
        cudaStreamSynchronize(p->stream);
    }
    if (p->plain) {
        p->h_off = off;
        if ((e = cudaMalloc(&p->d_pgrid, sizeof(float) * NF * NF)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_pbuf, 2 * sizeof(float) * NF * NF)) != cudaSuccess) {
            enufft_status st = cuda_fail(nullptr, e, "plan_create: plain-path scratch");
            enufft_plan_destroy(p);
            return st;
        }
        p->n_fused = 0;
        if (o.autotune && n_cells > 0 && !p->lbatches.empty()) {
            const std::string key = tune_key(p, o, NF, W);
            enufft_tuning t;
            if (!(o.tune_cache && tune_cache_get(o.tune_cache, key, &t) &&
                  (t.large_tile == 16 || t.large_tile == 32 || t.large_tile == 64))) {
                const enufft_status st = tune_large_tile(p, off, &t);
                if (st != ENUFFT_OK) {
                    enufft_plan_destroy(p);
                    return st;
                }
                cudaMemsetAsync(p->d_ctr + 2, 0, sizeof(unsigned), p->stream);   // the trial runs leave no status
                cudaStreamSynchronize(p->stream);
                if (o.tune_cache) tune_cache_put(o.tune_cache, key, t);   // best effort
            }
            p->tuned = true;
            p->tuning = t;
            p->lt = t.large_tile;
        }
        *out = p;
        return ENUFFT_OK;
    }
    if (p->large) {
        // batches of consecutive cells with bounded record and grid scratch; bin/scatter blocks
        std::vector<int4> blocks, work;
        std::vector<int2> cellblk(std::max<int64_t>(n_cells, 1));
        int64_t max_pts = 0;
        int max_blocks = 0;
        size_t max_work = 0;
        for (int64_t c = 0; c < n_cells;) {
            enufft_plan_s::LBatch b{(int)c, 0, (int)blocks.size(), 0, 0, 0, off[c]};
            while (c < n_cells && b.ncells < kLargeBatchCells &&
                   (b.ncells == 0 || off[c + 1] - b.p0 <= kLargeBatchPoints)) {
                const int first = (int)blocks.size() - b.block0;
                for (int64_t q = off[c]; q < off[c + 1]; q += kLBinBlock)
                    blocks.push_back(make_int4(b.ncells, (int)(q - b.p0), (int)std::min<int64_t>(off[c + 1] - b.p0, q - b.p0 + kLBinBlock), 0));
                cellblk[c] = make_int2(first, (int)blocks.size() - b.block0 - first);
                ++b.ncells;
                ++c;
            }
            b.nblocks = (int)blocks.size() - b.block0;
            // spread work items: cells of more than kLSplitPoints samples in parts, largest cells first
            std::vector<int> byq(b.ncells);
            std::iota(byq.begin(), byq.end(), 0);
            std::stable_sort(byq.begin(), byq.end(), [&](int u, int v) {
                return off[b.cell0 + u + 1] - off[b.cell0 + u] > off[b.cell0 + v + 1] - off[b.cell0 + v];
            });
            b.work0 = (int)work.size();
            for (int u : byq) {
                const int64_t qn = off[b.cell0 + u + 1] - off[b.cell0 + u];
                const int parts = (int)std::max<int64_t>(1, (qn + kLSplitPoints - 1) / kLSplitPoints);
                for (int k = 0; k < parts; ++k) work.push_back(make_int4(u, k, parts, 0));
            }
            b.nwork = (int)work.size() - b.work0;
            max_work = std::max(max_work, (size_t)b.nwork);
            max_pts = std::max<int64_t>(max_pts, off[c] - b.p0);
            max_blocks = std::max(max_blocks, b.nblocks);
            p->lmax_cells = std::max(p->lmax_cells, b.ncells);
            p->lbatches.push_back(b);
        }
        if (max_pts > 0x7fffffff) {
            enufft_plan_destroy(p);
            return fail(nullptr, ENUFFT_ERR_UNSUPPORTED, "plan_create: a cell has more than 2^31 samples");
        }
        const size_t mc = std::max(1, p->lmax_cells);
        if ((e = cudaMalloc(&p->d_lblocks, sizeof(int4) * std::max<size_t>(blocks.size(), 1))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lcellblk, sizeof(int2) * cellblk.size())) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lwork, sizeof(int4) * std::max<size_t>(work.size(), 1))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lblk_off, sizeof(int) * (kLTilesMax + 1) * std::max(max_blocks, 1))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lblk_abs, sizeof(float) * kLTilesMax * std::max(max_blocks, 1))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lrec, sizeof(float4) * std::max<int64_t>(max_pts, 1))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lgrid, sizeof(unsigned long long) * kLNF * kLNF * mc)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lexp, sizeof(int) * mc)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lpartial, sizeof(double) * 3 * std::max<size_t>(max_work, 1))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_lspec, sizeof(double) * 2 * std::max<int64_t>(n_cells, 1))) != cudaSuccess) {
            enufft_status st = cuda_fail(nullptr, e, "plan_create: large-route scratch");
            enufft_plan_destroy(p);
            return st;
        }
        if ((!blocks.empty() && (e = cudaMemcpyAsync(p->d_lblocks, blocks.data(), sizeof(int4) * blocks.size(),
                                                     cudaMemcpyHostToDevice, p->stream)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(p->d_lcellblk, cellblk.data(), sizeof(int2) * cellblk.size(), cudaMemcpyHostToDevice,
                                 p->stream)) != cudaSuccess ||
            (!work.empty() && (e = cudaMemcpyAsync(p->d_lwork, work.data(), sizeof(int4) * work.size(),
                                                   cudaMemcpyHostToDevice, p->stream)) != cudaSuccess)) {
            enufft_status st = cuda_fail(nullptr, e, "plan_create: block table");
            enufft_plan_destroy(p);
            return st;
        }
        cudaStreamSynchronize(p->stream);
        if ((e = large_prepare(p->P)) != cudaSuccess) {
            enufft_status st = cuda_fail(nullptr, e, "plan_create: large-route kernel attributes");
            enufft_plan_destroy(p);
            return st;
        }
        p->n_fused = 0;
        if (o.autotune && n_cells > 0 && !p->lbatches.empty()) {
            const std::string key = tune_key(p, o, NF, W);
            enufft_tuning t;
            if (!(o.tune_cache && tune_cache_get(o.tune_cache, key, &t) &&
                  (t.large_tile == 16 || t.large_tile == 32 || t.large_tile == 64))) {
                const enufft_status st = tune_large_tile(p, off, &t);
                if (st != ENUFFT_OK) {
                    enufft_plan_destroy(p);
                    return st;
                }
                cudaMemsetAsync(p->d_ctr + 2, 0, sizeof(unsigned), p->stream);   // the trial runs leave no status
                cudaStreamSynchronize(p->stream);
                if (o.tune_cache) tune_cache_put(o.tune_cache, key, t);   // best effort
            }
            p->tuned = true;
            p->tuning = t;
            p->lt = t.large_tile;
        }
        *out = p;
        return ENUFFT_OK;
    }
    if ((p->n_tc > 0 || (o.autotune && o.tc_max_points > 0)) && (e = tc_prepare()) != cudaSuccess) {
        enufft_status st = cuda_fail(nullptr, e, "plan_create: tensor-core kernel attributes");
        enufft_plan_destroy(p);
        return st;
    }
    e = fused_prepare(p->dbl, NF, W, &p->fwd_per_sm, &p->adj_per_sm);
    if (e != cudaSuccess || p->fwd_per_sm < 1 || p->adj_per_sm < 1) {
        enufft_status st = e != cudaSuccess ? cuda_fail(nullptr, e, "plan_create: kernel attributes")
                                            : fail(nullptr, ENUFFT_ERR_UNSUPPORTED, "plan_create: kernel does not fit an SM");
        enufft_plan_destroy(p);
        return st;
    }
    p->fwd_grid_per_sm = p->fwd_per_sm;
    if (o.autotune && !p->dbl && n_cells > 0) {
        const std::string key = tune_key(p, o, NF, W);
        enufft_tuning t;
        if (!(o.tune_cache && tune_cache_get(o.tune_cache, key, &t))) {
            std::vector<int64_t> q(n_cells);
            for (int64_t j = 0; j < n_cells; ++j) q[j] = off[j + 1] - off[j];
            std::nth_element(q.begin(), q.begin() + n_cells / 2, q.end());
            TuneEnv env{p->d_cells, (int)n_cells, p->P, NF, W, p->poly, p->beta, p->inv_phi, p->d_twiddle,
                        p->num_sms, p->fwd_per_sm, p->d_ctr + 2, p->stream, o.tc_max_points,
                        (int)std::min<int64_t>(q[n_cells / 2], 1 << 20)};
            if ((e = autotune_run(env, &t)) != cudaSuccess) {
                enufft_status st = cuda_fail(nullptr, e, "plan_create: autotune");
                enufft_plan_destroy(p);
                return st;
            }
            if (o.tune_cache) tune_cache_put(o.tune_cache, key, t);   // best effort: an unwritable cache is skipped
        }
        p->tuned = true;
        p->tuning = t;
        p->fwd_grid_per_sm = std::max(1, std::min(t.fused_blocks_per_sm, p->fwd_per_sm));
        p->tc_threshold = std::min(t.tc_max_points, o.tc_max_points);
        p->n_tc = 0;
        if (p->tc_threshold > 0)
            for (int64_t j = 0; j < n_cells; ++j)
                if (off[j + 1] - off[j] <= p->tc_threshold) ++p->n_tc;
        p->n_fused = (int)(n_cells - p->n_tc);
    }
    *out = p;
    return ENUFFT_OK;
}

enufft_status enufft_get_tuning(enufft_plan p, enufft_tuning* out) {
    if (!p || !out) return fail(p, ENUFFT_ERR_ARG, "get_tuning: NULL argument");
    if (!p->tuned) return fail(p, ENUFFT_ERR_ARG, "get_tuning: the plan was not tuned");
    *out = p->tuning;
    return ENUFFT_OK;
}

enufft_status enufft_get_plan_info(enufft_plan p, enufft_plan_info* info) {
    if (!p || !info) return fail(p, ENUFFT_ERR_ARG, "get_plan_info: NULL argument");
    info->modes = p->P;
    info->fine_grid = p->NF;
    info->kernel_width = p->W;
    info->beta = p->beta;
    info->oversamp_effective = p->sigma_eff;
    info->n_cells = p->n_cells;
    info->n_points = p->n_points;
    info->cells_fused = p->n_fused;
    info->cells_tensor = p->n_tc;
    info->cells_large = p->large ? p->n_cells : 0;
    info->precision = (int)p->opts.prec;
    info->cells_plain = p->plain ? p->n_cells : 0;
    info->kernel = (int)p->opts.kernel;
    info->frame = (int)p->opts.frame;
    info->tc_max_points = p->n_tc > 0 || p->tuned ? p->tc_threshold : 0;
    info->autotuned = p->tuned ? 1 : 0;
    info->fused_blocks_per_sm = p->fwd_grid_per_sm;
    info->large_tile = p->large ? p->lt : 0;
    int64_t k = 0;
    if (p->plain) {
        for (int64_t j = 0; j < p->n_cells; ++j) k += p->h_off[j + 1] > p->h_off[j] ? 4 : 3;
        k += 2;   // EMS ranking + finish
    } else if (p->large) {
        for (const auto& b : p->lbatches) k += b.ncells > 0 ? (b.nblocks > 0 ? 4 : 3) : 0;   // sort, scale, spread, FFT
        k += 1;   // EMS finish
    } else {
        k = (p->n_fused > 0) + (p->n_tc > 0) + 1;   // fused transform, tensor-core direct sum, EMS finish
    }
    if (p->edge && p->n_points > 0) k += 1;   // local coordinates of the samples
    info->kernels_per_type1_ems = p->n_cells > 0 ? k : 0;
    return ENUFFT_OK;
}

enufft_status enufft_set_stream(enufft_plan p, void* s) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "set_stream: NULL plan");
    p->stream = (cudaStream_t)s;
    return ENUFFT_OK;
}

enufft_status enufft_selftest_wait_timeout(enufft_plan p, unsigned polls) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "selftest_wait_timeout: NULL plan");
    if (polls < 1 || polls > (1u << 17)) return fail(p, ENUFFT_ERR_ARG, "selftest_wait_timeout: polls must be in [1, 2^17]");
    cudaSetDevice(p->device);
    cudaError_t e = launch_wait_timeout(polls, p->d_ctr + 2, p->stream);
    return e == cudaSuccess ? ENUFFT_OK : cuda_fail(p, e, "selftest_wait_timeout: launch");
}

enufft_status enufft_sync_status(enufft_plan p) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "sync_status: NULL plan");
    unsigned st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, p->d_ctr + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "sync_status");
    if (st) {
        cudaMemsetAsync(p->d_ctr + 2, 0, sizeof(unsigned), p->stream);
        cudaStreamSynchronize(p->stream);
        std::string m = "device status:";
        if (st & ST_NONFINITE) m += " non-finite sample(s) skipped;";
        if (st & ST_BADCELL) m += " degenerate cell polygon(s);";
        if (st & ST_TIMEOUT) m += " bounded wait expired;";
        if (st & ST_MOVED) m += " edge frame: sample(s) placed at the cell centroid (no binary32 point inside the window);";
        return fail(p, (st & ST_TIMEOUT) ? ENUFFT_ERR_TIMEOUT : ENUFFT_ERR_DEVICE, m);
    }
    return ENUFFT_OK;
}

enufft_status enufft_plan_sync_status(enufft_plan p) { return enufft_sync_status(p); }

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// execution
// ------------------------------------------------------------------------------------------------
static bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

static enufft_status check_ems_params(enufft_plan p, const enufft_ems_params* prm) {
    if (!prm) return fail(p, ENUFFT_ERR_ARG, "ems: params is NULL");
    if (prm->k_max < 1 || prm->k_max > kEmsMaxK) return fail(p, ENUFFT_ERR_ARG, "ems: k_max must be in [1, 64]");
    if (prm->k_min < 0 || prm->k_min > prm->k_max) return fail(p, ENUFFT_ERR_ARG, "ems: k_min must be in [0, k_max]");
    if (!(prm->delta > 0.0)) return fail(p, ENUFFT_ERR_ARG, "ems: delta must be positive");
    return ENUFFT_OK;
}

static EmsArgs make_ems(const enufft_ems_params* prm, const double* W, int per_cell, int32_t* ks, int32_t* sel,
                        double* ret) {
    EmsArgs a;
    a.k_min = prm->k_min;
    a.k_max = prm->k_max;
    a.alpha_min = prm->alpha_min;
    a.alpha_max = prm->alpha_max;
    a.delta = prm->delta;
    a.w1 = prm->w1;
    a.w2 = prm->w2;
    a.sum_over = prm->sum_over ? 1 : 0;
    a.include_dc = prm->include_dc ? 1 : 0;
    a.W = W;
    a.w_per_cell = per_cell ? 1 : 0;
    a.kstar = ks;
    a.sel = sel;
    a.retained = ret;
    return a;
}

// stand-alone EMS on coefficients in global memory: ranking kernel, then the per-cell finish
static enufft_status launch_ems(enufft_plan p, const void* d_coeffs, const EmsArgs& ea) {
    const size_t smem = ems_smem_bytes(16, ea.k_max);
    const int grid = (int)std::min<int64_t>(p->n_cells, (int64_t)p->num_sms * 4);
    const int half = p->P / 2, lim = half - 1;
    const int J = (lim > 0 ? lim * (2 * lim + 2) : 0) + 1;
    const bool big = J > 512 * 4;   // candidates per thread of the 512-thread ranking block
    const EmsScratch sc = p->ems_scratch;
    if (p->dbl) {
        if (big) ems_rank_kernel<double, 16><<<grid, 512, smem, p->stream>>>((const cplx<double>*)d_coeffs, p->P, p->n_cells, ea, sc);
        else ems_rank_kernel<double, 4><<<grid, 512, smem, p->stream>>>((const cplx<double>*)d_coeffs, p->P, p->n_cells, ea, sc);
    } else {
        if (big) ems_rank_kernel<float, 16><<<grid, 512, smem, p->stream>>>((const cplx<float>*)d_coeffs, p->P, p->n_cells, ea, sc);
        else ems_rank_kernel<float, 4><<<grid, 512, smem, p->stream>>>((const cplx<float>*)d_coeffs, p->P, p->n_cells, ea, sc);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p, e, "ems: launch");
    ems_finish_kernel<<<(unsigned)((p->n_cells + 127) / 128), 128, 0, p->stream>>>(p->n_cells, ea, sc);
    e = cudaGetLastError();
    return e == cudaSuccess ? ENUFFT_OK : cuda_fail(p, e, "ems: finish launch");
}

// the batches [0, nbatch) of the large route with tile side lt
static enufft_status run_large_batches(enufft_plan p, const void* x, const void* y, const void* h, const void* w,
                                       void* coeffs, const EmsArgs* ems, int lt, size_t nbatch) {
    LargeArgs la;
    memset(&la, 0, sizeof(la));
    la.x = (const float*)x;
    la.y = (const float*)y;
    la.h = (const float*)h;
    la.w = (const float*)w;
    la.cells = p->d_cells;
    la.blk_off = p->d_lblk_off;
    la.blk_abs = p->d_lblk_abs;
    la.rec = p->d_lrec;
    la.grid = p->d_lgrid;
    la.cell_exp = p->d_lexp;
    la.status = p->d_ctr + 2;
    la.poly = p->poly;
    la.W = p->W;
    LargeFftArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.grid = reinterpret_cast<const long long*>(p->d_lgrid);
    fa.cell_exp = p->d_lexp;
    fa.P = p->P;
    fa.coeffs = (float*)coeffs;
    fa.twiddle = (const cplx<float>*)p->d_twiddle;
    for (int k = 0; k <= p->P / 2; ++k) fa.inv_phi[k] = (float)p->inv_phi[k];
    fa.do_ems = ems ? 1 : 0;
    if (ems) fa.ems = *ems;
    fa.ems_out = p->ems_scratch;
    for (size_t bi = 0; bi < nbatch && bi < p->lbatches.size(); ++bi) {
        const auto& b = p->lbatches[bi];
        la.cell0 = fa.cell0 = b.cell0;
        la.ncells = fa.ncells = b.ncells;
        la.p0 = b.p0;
        la.blocks = p->d_lblocks + b.block0;
        la.cell_blocks = p->d_lcellblk + b.cell0;
        la.work = p->d_lwork + b.work0;
        cudaError_t e = cudaMemsetAsync(p->d_lgrid, 0, sizeof(unsigned long long) * kLNF * kLNF * (size_t)b.ncells,
                                        p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "type1 (large): memset");
        e = large_run_batch(la, std::max(b.nblocks, 0), b.nwork, fa, p->W, lt, std::min(b.ncells, p->num_sms),
                            p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "type1 (large): launch");
    }
    if (ems) {
        ems_finish_kernel<<<(unsigned)((p->n_cells + 127) / 128), 128, 0, p->stream>>>(p->n_cells, *ems, p->ems_scratch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(p, e, "type1_ems (large): finish launch");
    }
    return ENUFFT_OK;
}

static enufft_status run_type1_large(enufft_plan p, const void* x, const void* y, const void* h, const void* w,
                                     void* coeffs, const EmsArgs* ems) {
    return run_large_batches(p, x, y, h, w, coeffs, ems, p->lt, p->lbatches.size());
}

// Tile side of the large route by measurement (opts.autotune): the plan's first batch with
// synthetic samples (uniform over each cell's window) run with tiles of 16, 32 and 64; the record
// keeps the sides tried in ladder[] and the route's ns per sample with each in ns_fused[].
static enufft_status tune_large_tile(enufft_plan p, const std::vector<int64_t>& off, enufft_tuning* t) {
    memset(t, 0, sizeof(*t));
    t->fused_blocks_per_sm = 1;
    t->large_tile = kLT;
    const auto& b = p->lbatches[0];
    const int64_t npts = off[b.cell0 + b.ncells] - b.p0;
    if (npts <= 0) return ENUFFT_OK;
    float *x = nullptr, *y = nullptr, *h = nullptr, *w = nullptr;
    void* co = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    enufft_status st = ENUFFT_OK;
    if ((e = cudaMalloc(&x, 4 * (size_t)npts)) != cudaSuccess || (e = cudaMalloc(&y, 4 * (size_t)npts)) != cudaSuccess ||
        (e = cudaMalloc(&h, 4 * (size_t)npts)) != cudaSuccess || (e = cudaMalloc(&w, 4 * (size_t)npts)) != cudaSuccess ||
        (e = cudaMalloc(&co, sizeof(cplx<float>) * (size_t)p->P * p->P * (b.cell0 + b.ncells))) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
        (e = large_tune_samples(p->d_cells + b.cell0, p->d_offsets + b.cell0, b.p0, b.ncells, x, y, h, w,
                                p->stream)) != cudaSuccess) {
        st = cuda_fail(nullptr, e, "plan_create: tile tuning");
    } else {
        double best = 1e30;
        const int sides[3] = {16, 32, 64};
        t->n_ladder = 3;
        for (int i = 0; i < 3 && st == ENUFFT_OK; ++i) {
            double ms_best = 1e30;
            for (int rep = 0; rep < 3 && st == ENUFFT_OK; ++rep) {   // a warm-up, then the best of two
                cudaEventRecord(e0, p->stream);
                st = run_large_batches(p, x, y, h, w, co, nullptr, sides[i], 1);
                cudaEventRecord(e1, p->stream);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) st = cuda_fail(nullptr, e, "plan_create: tile tuning");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_best = std::min(ms_best, (double)ms);
            }
            t->ladder[i] = sides[i];
            t->ns_fused[i] = ms_best * 1e6 / (double)npts;
            if (ms_best < best) {
                best = ms_best;
                t->large_tile = sides[i];
            }
        }
        if (st != ENUFFT_OK) st = fail(nullptr, st, std::string("plan_create: tile tuning: ") + p->err);
    }
    cudaFree(x);
    cudaFree(y);
    cudaFree(h);
    cudaFree(w);
    cudaFree(co);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

static enufft_status run_type1_plain(enufft_plan p, const void* x, const void* y, const void* h, const void* w,
                                     void* coeffs, const EmsArgs* ems) {
    PlainRun r;
    r.x = (const float*)x;
    r.y = (const float*)y;
    r.h = (const float*)h;
    r.w = (const float*)w;
    r.h_off = p->h_off.data();
    r.n_cells = p->n_cells;
    r.cells = p->d_cells;
    r.NF = p->NF;
    r.W = p->W;
    r.P = p->P;
    r.beta = (float)p->beta;
    r.kind = p->poly.kind;
    r.inv_norm = (float)p->poly.inv_norm;
    r.inv_phi = p->inv_phi;
    r.twiddle = (const cplx<float>*)p->d_twiddle;
    r.grid = p->d_pgrid;
    r.buf = (cplx<float>*)p->d_pbuf;
    r.coeffs = (cplx<float>*)coeffs;
    r.status = p->d_ctr + 2;
    cudaError_t e = plain_run(r, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "type1 (plain): launch");
    return ems ? launch_ems(p, coeffs, *ems) : ENUFFT_OK;
}

template <typename T>
static enufft_status run_type1(enufft_plan p, const void* x, const void* y, const void* h, const void* w,
                               void* coeffs, const EmsArgs* ems) {
    if (p->plain) return run_type1_plain(p, x, y, h, w, coeffs, ems);
    if (p->large) return run_type1_large(p, x, y, h, w, coeffs, ems);
    FwdArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.x = (const T*)x;
    a.y = (const T*)y;
    a.h = (const T*)h;
    a.w = (const T*)w;
    a.coeffs = (T*)coeffs;
    a.offsets = p->d_offsets;
    a.cells = p->d_cells;
    a.order = p->d_order;
    a.n_work = p->n_fused;
    a.P = p->P;
    a.ticket = p->d_ctr + 0;
    a.status = p->d_ctr + 2;
    a.twiddle = (const cplx<T>*)p->d_twiddle;
    for (int k = 0; k <= p->P / 2; ++k) a.inv_phi[k] = (T)p->inv_phi[k];
    a.poly = p->poly;
    a.beta = p->beta;
    a.do_ems = ems ? 1 : 0;
    if (ems) a.ems = *ems;
    a.ems_out = p->ems_scratch;
    cudaError_t e = cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if (p->n_tc > 0) {
            TcLaunch l;
            l.x = (const float*)x;
            l.y = (const float*)y;
            l.h = (const float*)h;
            l.w = (const float*)w;
            l.offsets = p->d_offsets;
            l.cells = p->d_cells;
            l.list = p->d_order + p->n_fused;
            l.n_list = p->n_tc;
            l.P = p->P;
            l.NF = p->NF;
            l.num_sms = p->num_sms;
            l.coeffs = (cplx<float>*)coeffs;
            l.status = p->d_ctr + 2;
            l.ems = ems;
            l.ems_out = p->ems_scratch;
            e = launch_tc_nudft(l, p->stream);
            if (e != cudaSuccess) return cuda_fail(p, e, "type1: tensor-core launch");
        }
    }
    if (a.n_work > 0) {
        e = cudaMemsetAsync(p->d_ctr, 0, sizeof(unsigned), p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "type1: memset");
        const int grid = std::min<int64_t>(a.n_work, (int64_t)p->fwd_grid_per_sm * p->num_sms);
        e = launch_type1(a, p->NF, p->W, grid, p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "type1: launch");
    }
    if (ems) {
        ems_finish_kernel<<<(unsigned)((p->n_cells + 127) / 128), 128, 0, p->stream>>>(p->n_cells, *ems, p->ems_scratch);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(p, e, "type1_ems: finish launch");
    }
    return ENUFFT_OK;
}

// edge-aligned frame: the samples' local coordinates into plan scratch, and x, y pointed there
static enufft_status edge_prepass(enufft_plan p, const void*& x, const void*& y) {
    if (!p->edge || p->n_points == 0) return ENUFFT_OK;
    // one wave of persistent blocks: three resident per SM (the kernel's launch bound)
    const int grid = (int)std::min<int64_t>(p->n_cells, (int64_t)p->num_sms * 3);
    cudaError_t e = launch_edge_frame(p->dbl, x, y, p->d_offsets, p->d_cells, p->d_rot, p->n_cells, p->d_vx, p->d_vy,
                                      p->d_ctr + 2, grid, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "edge frame: launch");
    x = p->d_vx;
    y = p->d_vy;
    return ENUFFT_OK;
}

extern "C" {

enufft_status enufft_type1(enufft_plan p, const void* d_x, const void* d_y, const void* d_h, const void* d_w,
                           void* d_coeffs) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "type1: NULL plan");
    if (p->n_cells == 0) return ENUFFT_OK;
    if (!d_coeffs || (p->n_points > 0 && (!d_x || !d_y || !d_h || !d_w)))
        return fail(p, ENUFFT_ERR_ARG, "type1: NULL data pointer");
    if (!aligned16(d_coeffs)) return fail(p, ENUFFT_ERR_ARG, "type1: coeffs must be 16-byte aligned");
    cudaSetDevice(p->device);
    const enufft_status es = edge_prepass(p, d_x, d_y);
    if (es != ENUFFT_OK) return es;
    return p->dbl ? run_type1<double>(p, d_x, d_y, d_h, d_w, d_coeffs, nullptr)
                  : run_type1<float>(p, d_x, d_y, d_h, d_w, d_coeffs, nullptr);
}

enufft_status enufft_type1_ems(enufft_plan p, const void* d_x, const void* d_y, const void* d_h, const void* d_w,
                               void* d_coeffs, const double* d_mode_weights, int per_cell,
                               const enufft_ems_params* prm, int32_t* d_kstar, int32_t* d_sel,
                               double* d_retained) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "type1_ems: NULL plan");
    enufft_status st = check_ems_params(p, prm);
    if (st != ENUFFT_OK) return st;
    if (p->n_cells == 0) return ENUFFT_OK;
    if (!d_coeffs || !d_kstar || !d_sel || !d_retained || (p->n_points > 0 && (!d_x || !d_y || !d_h || !d_w)))
        return fail(p, ENUFFT_ERR_ARG, "type1_ems: NULL data pointer");
    if (!aligned16(d_coeffs)) return fail(p, ENUFFT_ERR_ARG, "type1_ems: coeffs must be 16-byte aligned");
    cudaSetDevice(p->device);
    st = edge_prepass(p, d_x, d_y);
    if (st != ENUFFT_OK) return st;
    const EmsArgs ea = make_ems(prm, d_mode_weights, per_cell, d_kstar, d_sel, d_retained);
    return p->dbl ? run_type1<double>(p, d_x, d_y, d_h, d_w, d_coeffs, &ea)
                  : run_type1<float>(p, d_x, d_y, d_h, d_w, d_coeffs, &ea);
}

static bool same_key(const enufft_plan_s::GraphKey& a, const enufft_plan_s::GraphKey& b) {
    return a.x == b.x && a.y == b.y && a.h == b.h && a.w == b.w && a.coeffs == b.coeffs && a.mw == b.mw &&
           a.per_cell == b.per_cell && a.kstar == b.kstar && a.sel == b.sel && a.ret == b.ret &&
           a.prm.k_min == b.prm.k_min && a.prm.k_max == b.prm.k_max && a.prm.alpha_min == b.prm.alpha_min &&
           a.prm.alpha_max == b.prm.alpha_max && a.prm.delta == b.prm.delta && a.prm.w1 == b.prm.w1 &&
           a.prm.w2 == b.prm.w2 && a.prm.sum_over == b.prm.sum_over && a.prm.include_dc == b.prm.include_dc;
}

enufft_status enufft_type1_ems_graph(enufft_plan p, const void* d_x, const void* d_y, const void* d_h,
                                     const void* d_w, void* d_coeffs, const double* d_mode_weights, int per_cell,
                                     const enufft_ems_params* prm, int32_t* d_kstar, int32_t* d_sel,
                                     double* d_retained) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "type1_ems_graph: NULL plan");
    enufft_status st = check_ems_params(p, prm);
    if (st != ENUFFT_OK) return st;
    if (p->n_cells == 0) return ENUFFT_OK;
    if (!d_coeffs || !d_kstar || !d_sel || !d_retained || (p->n_points > 0 && (!d_x || !d_y || !d_h || !d_w)))
        return fail(p, ENUFFT_ERR_ARG, "type1_ems_graph: NULL data pointer");
    if (!aligned16(d_coeffs)) return fail(p, ENUFFT_ERR_ARG, "type1_ems_graph: coeffs must be 16-byte aligned");
    cudaSetDevice(p->device);
    const enufft_plan_s::GraphKey key = {d_x, d_y, d_h, d_w, d_coeffs, d_mode_weights, per_cell, *prm,
                                         d_kstar, d_sel, d_retained};
    if (!p->gexec || !same_key(key, p->gkey)) {
        if (p->gexec) {
            cudaError_t e = cudaStreamSynchronize(p->stream);   // the old graph may still run
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
            if (e != cudaSuccess) return cuda_fail(p, e, "type1_ems_graph: synchronise");
        }
        cudaError_t e = cudaSuccess;
        if (!p->gstream) e = cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(p, e, "type1_ems_graph: stream");
        // capture on the plan's own stream (the caller's may be the legacy default stream, which
        // cannot be captured); the kernels are recorded, not run
        const cudaStream_t user = p->stream;
        p->stream = p->gstream;
        e = cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            p->stream = user;
            return cuda_fail(p, e, "type1_ems_graph: begin capture");
        }
        st = enufft_type1_ems(p, d_x, d_y, d_h, d_w, d_coeffs, d_mode_weights, per_cell, prm, d_kstar, d_sel,
                              d_retained);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(p->gstream, &graph);
        p->stream = user;
        if (st != ENUFFT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            p->gexec = nullptr;
            return cuda_fail(p, e, "type1_ems_graph: capture");
        }
        p->gkey = key;
    }
    cudaError_t e = cudaGraphLaunch(p->gexec, p->stream);
    return e == cudaSuccess ? ENUFFT_OK : cuda_fail(p, e, "type1_ems_graph: launch");
}

enufft_status enufft_ems(enufft_plan p, const void* d_coeffs, const double* d_mode_weights, int per_cell,
                         const enufft_ems_params* prm, int32_t* d_kstar, int32_t* d_sel, double* d_retained) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "ems: NULL plan");
    enufft_status st = check_ems_params(p, prm);
    if (st != ENUFFT_OK) return st;
    if (p->n_cells == 0) return ENUFFT_OK;
    if (!d_coeffs || !d_kstar || !d_sel || !d_retained) return fail(p, ENUFFT_ERR_ARG, "ems: NULL data pointer");
    cudaSetDevice(p->device);
    const EmsArgs ea = make_ems(prm, d_mode_weights, per_cell, d_kstar, d_sel, d_retained);
    return launch_ems(p, d_coeffs, ea);
}

enufft_status enufft_ems_backward(enufft_plan p, const void* d_coeffs, const double* d_mode_weights, int per_cell,
                                  const enufft_ems_params* prm, const int32_t* d_kstar, const int32_t* d_sel,
                                  const double* d_grad_power, void* d_grad_coeffs) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "ems_backward: NULL plan");
    enufft_status st = check_ems_params(p, prm);
    if (st != ENUFFT_OK) return st;
    if (p->n_cells == 0) return ENUFFT_OK;
    if (!d_coeffs || !d_kstar || !d_sel || !d_grad_power || !d_grad_coeffs)
        return fail(p, ENUFFT_ERR_ARG, "ems_backward: NULL data pointer");
    if (!aligned16(d_grad_coeffs)) return fail(p, ENUFFT_ERR_ARG, "ems_backward: grad_coeffs must be 16-byte aligned");
    cudaSetDevice(p->device);
    const int grid = (int)std::min<int64_t>(p->n_cells, (int64_t)p->num_sms * 8);
    if (p->dbl)
        ems_backward_kernel<double><<<grid, 256, 0, p->stream>>>((const cplx<double>*)d_coeffs, p->P, p->n_cells,
                                                               d_mode_weights, per_cell, prm->k_max, d_kstar, d_sel,
                                                               d_grad_power, (cplx<double>*)d_grad_coeffs);
    else
        ems_backward_kernel<float><<<grid, 256, 0, p->stream>>>((const cplx<float>*)d_coeffs, p->P, p->n_cells,
                                                              d_mode_weights, per_cell, prm->k_max, d_kstar, d_sel,
                                                              d_grad_power, (cplx<float>*)d_grad_coeffs);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ENUFFT_OK : cuda_fail(p, e, "ems_backward: launch");
}

}  // extern "C"

// adjoint / reconstruction of the n_f = 256 route, batch by batch (large_adj.cuh)
static enufft_status run_adjoint_large(enufft_plan p, const void* g, const void* x, const void* y, const void* h,
                                       const void* w, void* gh, void* gw, const AdjArgs<float>* recon) {
    LargeAdjFftArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.gcoef = (const float*)g;
    fa.mode = recon ? 1 : 0;
    fa.P = p->P;
    fa.grid = reinterpret_cast<float*>(p->d_lgrid);
    fa.spec = p->d_lspec;
    fa.twiddle = (const cplx<float>*)p->d_twiddle;
    for (int k = 0; k <= p->P / 2; ++k) fa.inv_phi[k] = (float)p->inv_phi[k];
    LargeInterpArgs ia;
    memset(&ia, 0, sizeof(ia));
    ia.x = (const float*)x;
    ia.y = (const float*)y;
    ia.h = (const float*)h;
    ia.w = (const float*)w;
    ia.offsets = p->d_offsets;
    ia.cells = p->d_cells;
    ia.grid = fa.grid;
    ia.mode = fa.mode;
    ia.grad_h = (float*)gh;
    ia.grad_w = (float*)gw;
    ia.partial = p->d_lpartial;
    ia.status = p->d_ctr + 2;
    ia.poly = p->poly;
    if (recon) {
        fa.kstar = recon->kstar;
        fa.sel = recon->sel;
        fa.k_max = recon->k_max;
        ia.hrec = recon->hrec;
    }
    for (const auto& b : p->lbatches) {
        fa.cell0 = ia.cell0 = b.cell0;
        fa.ncells = b.ncells;
        ia.work = p->d_lwork + b.work0;
        cudaError_t e = large_run_adjoint_batch(fa, ia, b.nwork, p->W, std::min(b.ncells, p->num_sms),
                                                recon ? recon->stats : nullptr, p->d_cells, p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "adjoint (large): launch");
    }
    return ENUFFT_OK;
}

template <typename T>
static enufft_status run_adjoint(enufft_plan p, const void* g, const void* x, const void* y, const void* h,
                                 const void* w, void* gh, void* gw, const AdjArgs<T>* recon = nullptr) {
    if constexpr (sizeof(T) == 4) {
        if (p->large) return run_adjoint_large(p, g, x, y, h, w, gh, gw, recon);
    }
    AdjArgs<T> a;
    memset(&a, 0, sizeof(a));
    if (recon) a = *recon;
    a.x = (const T*)x;
    a.y = (const T*)y;
    a.h = (const T*)h;
    a.w = (const T*)w;
    a.gcoef = (const T*)g;
    a.grad_h = (T*)gh;
    a.grad_w = (T*)gw;
    a.offsets = p->d_offsets;
    a.cells = p->d_cells;
    a.order = p->d_order;
    a.n_work = (int)p->n_cells;   // the adjoint of every cell, whichever route made its coefficients
    a.P = p->P;
    a.ticket = p->d_ctr + 1;
    a.status = p->d_ctr + 2;
    a.twiddle = (const cplx<T>*)p->d_twiddle;
    for (int k = 0; k <= p->P / 2; ++k) a.inv_phi[k] = (T)p->inv_phi[k];
    a.poly = p->poly;
    a.beta = p->beta;
    if (a.n_work == 0) return ENUFFT_OK;
    cudaError_t e = cudaMemsetAsync(p->d_ctr + 1, 0, sizeof(unsigned), p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "type1_backward: memset");
    const int grid = std::min<int64_t>(a.n_work, (int64_t)p->adj_per_sm * p->num_sms);
    e = launch_adjoint(a, p->NF, p->W, grid, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "type1_backward: launch");
    return ENUFFT_OK;
}

template <typename T>
static enufft_status run_reconstruct(enufft_plan p, const void* coeffs, const int32_t* kstar, const int32_t* sel,
                                     int k_max, const void* x, const void* y, const void* h, const void* w, void* hrec,
                                     double* stats) {
    AdjArgs<T> r;
    memset(&r, 0, sizeof(r));
    r.mode = 1;
    r.kstar = kstar;
    r.sel = sel;
    r.k_max = k_max;
    r.hrec = (T*)hrec;
    r.stats = stats;
    return run_adjoint<T>(p, coeffs, x, y, h, w, nullptr, nullptr, &r);
}

extern "C" enufft_status enufft_voronoi_weights(enufft_plan p, const void* d_x, const void* d_y, int ng, void* d_w) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "voronoi_weights: NULL plan");
    if (ng < 2 || ng > 1024) return fail(p, ENUFFT_ERR_ARG, "voronoi_weights: ng must be in [2, 1024]");
    if (p->n_cells == 0) return ENUFFT_OK;
    if (p->n_points > 0 && (!d_x || !d_y || !d_w)) return fail(p, ENUFFT_ERR_ARG, "voronoi_weights: NULL data pointer");
    if (p->dbl) return fail(p, ENUFFT_ERR_UNSUPPORTED, "voronoi_weights: binary32 samples only");
    if (p->edge) return fail(p, ENUFFT_ERR_UNSUPPORTED, "voronoi_weights: not built for edge-frame plans");
    cudaSetDevice(p->device);
    cudaError_t e = launch_voronoi((const float*)d_x, (const float*)d_y, p->d_offsets, p->d_cells, (int)p->n_cells, ng,
                                   (float*)d_w, p->d_ctr + 2, p->num_sms, p->stream);
    return e == cudaSuccess ? ENUFFT_OK : cuda_fail(p, e, "voronoi_weights: launch");
}

extern "C" enufft_status enufft_reconstruct(enufft_plan p, const void* d_coeffs, const int32_t* d_kstar,
                                            const int32_t* d_sel, int k_max, const void* d_x, const void* d_y,
                                            const void* d_h, const void* d_w, void* d_hrec, double* d_stats) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "reconstruct: NULL plan");
    if (k_max < 1 || k_max > kEmsMaxK) return fail(p, ENUFFT_ERR_ARG, "reconstruct: k_max must be in [1, 64]");
    if (p->n_cells == 0) return ENUFFT_OK;
    if (!d_coeffs || !d_kstar || !d_sel || !d_stats || (p->n_points > 0 && (!d_x || !d_y || !d_h || !d_w)))
        return fail(p, ENUFFT_ERR_ARG, "reconstruct: NULL data pointer");
    if (!aligned16(d_coeffs)) return fail(p, ENUFFT_ERR_ARG, "reconstruct: coeffs must be 16-byte aligned");
    if (p->plain) return fail(p, ENUFFT_ERR_UNSUPPORTED, "reconstruct: not built for plain FP32 plans");
    cudaSetDevice(p->device);
    const enufft_status es = edge_prepass(p, d_x, d_y);
    if (es != ENUFFT_OK) return es;
    return p->dbl ? run_reconstruct<double>(p, d_coeffs, d_kstar, d_sel, k_max, d_x, d_y, d_h, d_w, d_hrec, d_stats)
                  : run_reconstruct<float>(p, d_coeffs, d_kstar, d_sel, k_max, d_x, d_y, d_h, d_w, d_hrec, d_stats);
}

extern "C" enufft_status enufft_type1_backward(enufft_plan p, const void* d_grad_coeffs, const void* d_x,
                                               const void* d_y, const void* d_h, const void* d_w, void* d_grad_h,
                                               void* d_grad_w) {
    if (!p) return fail(nullptr, ENUFFT_ERR_ARG, "type1_backward: NULL plan");
    if (p->n_cells == 0) return ENUFFT_OK;
    if (!d_grad_coeffs || (p->n_points > 0 && (!d_x || !d_y || !d_h || !d_w)))
        return fail(p, ENUFFT_ERR_ARG, "type1_backward: NULL data pointer");
    if (!aligned16(d_grad_coeffs)) return fail(p, ENUFFT_ERR_ARG, "type1_backward: grad_coeffs must be 16-byte aligned");
    if (p->plain) return fail(p, ENUFFT_ERR_UNSUPPORTED, "type1_backward: not built for plain FP32 plans");
    cudaSetDevice(p->device);
    const enufft_status es = edge_prepass(p, d_x, d_y);
    if (es != ENUFFT_OK) return es;
    return p->dbl ? run_adjoint<double>(p, d_grad_coeffs, d_x, d_y, d_h, d_w, d_grad_h, d_grad_w)
                  : run_adjoint<float>(p, d_grad_coeffs, d_x, d_y, d_h, d_w, d_grad_h, d_grad_w);
}
