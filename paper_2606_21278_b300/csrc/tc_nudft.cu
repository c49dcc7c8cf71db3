// tc_nudft.cu -- direct NUDFT of small cells on the tensor cores (Eq. discrete_quadrature as a
// dense contraction):
//
//   h^[n][m] = (1/|D|) sum_q win_q w_q h_q e^{-i k_n y'_q} e^{-i k_m x'_q},   k = 2 pi / L,
//
// i.e. D = A^T B with A[q][.] = c_q (e^{-i k_n y'_q})_n and B[q][.] = (e^{-i k_m x'_q})_m over the
// samples q of the cell.  Complex values are stacked as real features (rows 0..63 the real parts
// of modes -P/2 .. P/2-1, rows 64..127 the imaginary parts), so one 128 x 128 real product per
// 16 samples carries the whole P x P complex result (P <= 64):
//   Re h^ = D[re n][re m] - D[im n][im m],   Im h^ = D[re n][im m] + D[im n][re m].
// Each value is split into binary16 hi + lo and the product is accumulated in binary32 as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo * lo term is below 2^-22 of the scale).  The samples'
// weights are scaled by 1 / max |c| of the cell so that every operand lies in [-1, 1].
//
// The tensor core adds the products of every MMA to the binary32 accumulator without rounding to
// nearest, so the accumulator error grows with the number of MMAs it absorbs; each accumulator run
// is therefore limited to 256 samples (two banks of 128 TMEM columns alternate), and finished runs
// are added into the staged spectrum in shared memory with round-to-nearest binary32 additions.
//
// One CTA per cell at a time (two per SM), warp-specialised: two set-up warps, one per stage, each
// prepare every other chunk of samples (window, scaled weight, coordinates, unit phasor steps) with
// the samples of their next chunk already loaded; one warp issues the tcgen05 MMAs; eight operand
// warps turn each chunk of 32 samples into binary16 operands in shared memory (double buffered).
// The hand-offs are mbarriers with bounded waits (set-up ready, operands written, MMAs done), so
// the operand warps never wait on a block-wide barrier inside a cell.  The
// accumulator lives in tensor memory and is read back per run, combined through shared memory,
// written out and ranked for EMS (Sec. 2.2).
#include <cuda_fp16.h>

#include "ems.cuh"
#include "forward.cuh"
#include "internal.h"
#include "tc.cuh"

namespace enufft {

namespace {

constexpr int kFeatThreads = 256;                         // warps 0..7: operands, TMEM read-back
constexpr int kMmaWarp = kFeatThreads / 32;               // warp 8: MMA issue
constexpr int kPrepWarp0 = kMmaWarp + 1;                  // warps 9, 10: sample set-up of stage 0, 1
constexpr int kTcThreads = kFeatThreads + 3 * 32;
constexpr int kCh = 32;                                   // samples per chunk (K of one stage)
constexpr unsigned kOpBytes = kCh * tc::kTcFeat * 2;      // one operand (8 KB)
constexpr unsigned kStageBytes = 4 * kOpBytes;            // A_hi, A_lo, B_hi, B_lo
constexpr int kHS = 65;                                   // row stride (complex) of the staged spectrum
constexpr unsigned kSpecOff = 2 * kStageBytes;
constexpr unsigned kSpecBytes = 64 * kHS * 8;
constexpr int kPrepF = 9;                                 // per sample: c, tx hi/lo, ty hi/lo, x and y steps
constexpr unsigned kPrepOff = kSpecOff + kSpecBytes;
constexpr unsigned kPrepBytes = 2 * kPrepF * kCh * 4;
constexpr unsigned kEmsOff = kPrepOff + kPrepBytes;
constexpr unsigned kEmsBytes = (unsigned)((ems_smem_bytes(kTcThreads / 32, kEmsMaxK) + 15) / 16 * 16);
constexpr unsigned kMiscOff = kEmsOff + kEmsBytes;
constexpr unsigned kSmemBytes = kMiscOff + 128;
constexpr unsigned kWaitLimit = 1u << 22;
constexpr int kBlockChunks = 8;                           // chunks accumulated per TMEM run (256 samples)
constexpr unsigned kTmemCols = 256;                       // two 128-column accumulator banks
static_assert(kCh % 16 == 0 && tc::tc_off(127, kCh - 1) < kOpBytes, "operand layout");
static_assert(kFeatThreads == 8 * kCh, "one (sample, feature octet) task per operand thread and axis");

struct TcSpec {
    const cplx<float>* hs;
    int half;
    __device__ __forceinline__ cplx<float> get(int m, int n) const { return hs[(n + half) * kHS + (m + half)]; }
};

}  // namespace

struct TcArgs {
    const float* __restrict__ x;
    const float* __restrict__ y;
    const float* __restrict__ h;
    const float* __restrict__ w;
    const int64_t* __restrict__ offsets;
    const CellConst* __restrict__ cells;
    const int* __restrict__ list;     // cells of this route
    int n_list, P, NF;
    cplx<float>* __restrict__ coeffs;
    unsigned* status;
    int do_ems;
    EmsArgs ems;
    EmsScratch ems_out;
};

// c e^{-2 pi i m (t + 1/2)} for m = m0 .. m0 + 7 (t = th + tl, |t| <= 1/2; (wr, wi) = -e^{-2 pi i t}),
// zero beyond slot P unless FULL (P = 64).  The anchor m0 takes one fast sine/cosine of an argument
// reduced to [-pi, pi] (absolute error below 1e-6); the 7 rotations use the accurate step.
template <bool FULL>
__device__ __forceinline__ void tc_phasors(float th, float tl, float wr, float wi, float c, int m0, int slot0, int P,
                                           float (&re)[8], float (&im)[8]) {
    const float fm0 = (float)m0;
    const float p = fm0 * th;
    const float r = (p - rintf(p)) + __fmaf_rn(fm0, tl, __fmaf_rn(fm0, th, -p));
    float s0, c0;
    __sincosf(6.283185307179586f * r, &s0, &c0);
    const float sg = (m0 & 1) ? -c : c;
    float zr = sg * c0, zi = -sg * s0;     // c (-1)^{m0} e^{-2 pi i m0 t}
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool on = FULL || slot0 + j < P;
        re[j] = on ? zr : 0.0f;
        im[j] = on ? zi : 0.0f;
        const float nr = zr * wr - zi * wi, ni = zr * wi + zi * wr;
        zr = nr;
        zi = ni;
    }
}

// Setup of one sample (Sec. 2.1, App. A): window test, scaled weight c / max |c|, and the centred
// coordinates u / L of both axes as binary32 hi + lo and the unit steps -e^{-2 pi i u/L}; writes
// slot k of a prep buffer (zeros for absent, outside or non-finite samples; the latter also latch
// ST_NONFINITE).
__device__ __forceinline__ void tc_prep_sample(const FastFrame& ff, const CellConst& cc, bool present, float px,
                                               float py, float hv, float wv, float inv_cm, float inv_nf, float* pr,
                                               int k, unsigned* status) {
    float c = 0.0f, txh = 0.0f, txl = 0.0f, tyh = 0.0f, tyl = 0.0f;
    if (present) {
        if (!(isfinite(px) && isfinite(py))) {
            atomicOr(status, ST_NONFINITE);
        } else {
            float uxh, uxl, uyh, uyl;
            two_diff(px, ff.cxh, uxh, uxl);
            uxl = __fsub_rn(uxl, ff.cxl);
            two_diff(py, ff.cyh, uyh, uyl);
            uyl = __fsub_rn(uyl, ff.cyl);
            int win = window_f32(ff, cc.edge, uxh + uxl, uyh + uyl);
            if (win < 0) win = window_f64(cc, (double)px, (double)py);
            if (win) {
                const float cv = wv * hv * ff.inv_area;
                if (!isfinite(cv)) {
                    atomicOr(status, ST_NONFINITE);
                } else {
                    c = cv * inv_cm;
                    const float qx = uxh * ff.sch, qy = uyh * ff.sch;
                    txh = qx * inv_nf;
                    txl = (__fmaf_rn(uxh, ff.sch, -qx) + __fmaf_rn(uxh, ff.scl, uxl * ff.sch)) * inv_nf;
                    tyh = qy * inv_nf;
                    tyl = (__fmaf_rn(uyh, ff.sch, -qy) + __fmaf_rn(uyh, ff.scl, uyl * ff.sch)) * inv_nf;
                }
            }
        }
    }
    float sx, cx, sy, cy;
    sincospif(2.0f * (txh + txl), &sx, &cx);
    sincospif(2.0f * (tyh + tyl), &sy, &cy);
    pr[k] = c;
    pr[kCh + k] = txh;
    pr[2 * kCh + k] = txl;
    pr[3 * kCh + k] = tyh;
    pr[4 * kCh + k] = tyl;
    pr[5 * kCh + k] = -cx;
    pr[6 * kCh + k] = sx;
    pr[7 * kCh + k] = -cy;
    pr[8 * kCh + k] = sy;
}

// eight binary32 values -> binary16 hi and lo octets (16 bytes each)
__device__ __forceinline__ void tc_split8(const float (&v)[8], uint4& hi, uint4& lo) {
    unsigned hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __half2 hh = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
        hw[j] = *reinterpret_cast<const unsigned*>(&hh);
        lw[j] = *reinterpret_cast<const unsigned*>(&ll);
    }
    hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

__device__ __forceinline__ void feat_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kFeatThreads) : "memory"); }

// hs[n][m] += (D[re n][re m] - D[im n][im m], D[re n][im m] + D[im n][re m]) for one accumulator
// bank; taken by the 256 operand threads (TMEM lane quarter warp & 3, column half warp >> 2), in
// two passes of 16 columns
__device__ __forceinline__ void tc_flush(unsigned bank, cplx<float>* hs, int warp, int lane) {
    const int lg = warp & 3, chh = warp >> 2;
    const int row = 32 * lg + lane;
    feat_sync();   // earlier writes of hs by other operand threads are complete
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        const int c0 = 32 * chh + 16 * pass;
        const unsigned ta = bank + ((unsigned)(32 * lg) << 16) + c0;
        float vr[16], vi[16];
        tc::tmem_ld16(ta, vr);
        tc::tmem_ld16(ta + 64, vi);
        tc::tmem_ld_wait();
        cplx<float>* dst = hs + (row & 63) * kHS + c0;
        if (row < 64) {
#pragma unroll
            for (int j = 0; j < 16; ++j) dst[j] = cplx<float>{dst[j].re + vr[j], dst[j].im + vi[j]};
        }
        feat_sync();
        if (row >= 64) {
#pragma unroll
            for (int j = 0; j < 16; ++j) dst[j] = cplx<float>{dst[j].re - vi[j], dst[j].im + vr[j]};
        }
        feat_sync();
    }
    tc::fence_before_sync();
}

template <bool FULL>
__global__ void __launch_bounds__(kTcThreads, 2) tc_nudft_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tsmem[];
    unsigned char* smem = tsmem;
    cplx<float>* hs = reinterpret_cast<cplx<float>*>(smem + kSpecOff);
    float* prep = reinterpret_cast<float*>(smem + kPrepOff);
    unsigned char* ems_sm = smem + kEmsOff;
    unsigned long long* bar_mma = reinterpret_cast<unsigned long long*>(smem + kMiscOff);   // [2] MMAs done
    unsigned long long* bar_full = bar_mma + 2;                                              // [2] operands written
    unsigned long long* bar_prep = bar_mma + 4;                                              // [2] set-up ready
    unsigned* tbase = reinterpret_cast<unsigned*>(smem + kMiscOff + 48);
    float* red = reinterpret_cast<float*>(smem + kMiscOff + 64);   // 9 warps
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = a.P, half = P / 2;

    if (warp == 0) {
        tc::tmem_alloc(tc::smem_addr(tbase), kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(tc::smem_addr(&bar_mma[s]), 1);
            tc::mbar_init(tc::smem_addr(&bar_full[s]), kFeatThreads);
            tc::mbar_init(tc::smem_addr(&bar_prep[s]), 1);
        }
        tc::mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const unsigned tmem = *tbase;
    const unsigned sbase = tc::smem_addr(smem);
    const unsigned idesc = tc::idesc_f16_f32_mn(128, 128);
    unsigned g = 0;   // chunks of this CTA so far (stage = g & 1, use of the stage = g >> 1)

    for (int li = blockIdx.x; li < a.n_list; li += gridDim.x) {
        const int cell = a.list[li];
        const CellConst& cc = a.cells[cell];
        const int64_t q0 = a.offsets[cell], q1 = a.offsets[cell + 1];
        const bool valid = cc.valid != 0;
        // ---- the samples toward L2 ahead of use: this cell's coordinates when it is the CTA's first,
        // the next cell's four arrays always (the control warp's one-chunk lookahead then waits on
        // L2, not on DRAM)
        if (li == (int)blockIdx.x) {
            prefetch_l2(a.x, q0, q1, tid, kTcThreads);
            prefetch_l2(a.y, q0, q1, tid, kTcThreads);
        }
        if (li + (int)gridDim.x < a.n_list) {
            const int nc = a.list[li + gridDim.x];
            const int64_t n0 = a.offsets[nc], n1 = a.offsets[nc + 1];
            prefetch_l2(a.x, n0, n1, tid, kTcThreads);
            prefetch_l2(a.y, n0, n1, tid, kTcThreads);
            prefetch_l2(a.h, n0, n1, tid, kTcThreads);
            prefetch_l2(a.w, n0, n1, tid, kTcThreads);
        }
        // ---- scale: max |w h| / |D| over the cell (binary32)
        float cm = 0.0f;
        if (valid)
            for (int64_t q = q0 + tid; q < q1; q += kTcThreads) {
                const float v = fabsf(a.w[q] * a.h[q] * cc.inv_area);
                if (v <= 3.0e38f) cm = fmaxf(cm, v);
            }
        for (int o = 16; o; o >>= 1) cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
        if (lane == 0) red[warp] = cm;
        for (int i = tid; i < 64 * kHS; i += kTcThreads) hs[i] = cplx<float>{0.0f, 0.0f};
        __syncthreads();
        cm = 0.0f;
        for (int i = 0; i < kTcThreads / 32; ++i) cm = fmaxf(cm, red[i]);
        const float inv_cm = cm > 0.0f ? 1.0f / cm : 0.0f;
        const int nch = (valid && cm > 0.0f) ? (int)((q1 - q0 + kCh - 1) / kCh) : 0;

        if (warp == kMmaWarp) {
            // ---- MMA warp: the three split products of each chunk once its operands are written
            for (int ch = 0; ch < nch; ++ch) {
                const unsigned gc = g + ch, st = gc & 1u;
                if (!tc::mbar_wait(tc::smem_addr(&bar_full[st]), (gc >> 1) & 1u, kWaitLimit)) atomicOr(a.status, ST_TIMEOUT);
                tc::fence_after_sync();
                if (lane == 0) {
                    const unsigned s0 = sbase + st * kStageBytes;
                    const unsigned acc = tmem + 128u * ((ch / kBlockChunks) & 1);
                    const bool first = ch % kBlockChunks == 0;
#pragma unroll
                    for (int s = 0; s < kCh / 16; ++s) {
                        const uint64_t ah = tc::smem_desc(s0 + s * 4096, tc::kTcLbo, tc::kTcSbo);
                        const uint64_t al = tc::smem_desc(s0 + kOpBytes + s * 4096, tc::kTcLbo, tc::kTcSbo);
                        const uint64_t bh = tc::smem_desc(s0 + 2 * kOpBytes + s * 4096, tc::kTcLbo, tc::kTcSbo);
                        const uint64_t bl = tc::smem_desc(s0 + 3 * kOpBytes + s * 4096, tc::kTcLbo, tc::kTcSbo);
                        tc::mma_f16(acc, ah, bh, idesc, (!first || s > 0) ? 1u : 0u);
                        tc::mma_f16(acc, ah, bl, idesc, 1u);
                        tc::mma_f16(acc, al, bh, idesc, 1u);
                    }
                    tc::mma_commit(tc::smem_addr(&bar_mma[st]));
                }
                __syncwarp();
            }
        } else if (warp >= kPrepWarp0) {
            // ---- set-up warp of stage sp: chunks ch with (g + ch) & 1 == sp, each into the stage's
            // set-up buffer once the operand warps have written the chunk two before (which read it)
            const unsigned sp = (unsigned)(warp - kPrepWarp0);
            const FastFrame ff = fast_frame(cc);
            const float inv_nf = 1.0f / (float)a.NF;
            float rx = 0.f, ry = 0.f, rh = 0.f, rw = 0.f;
            bool rv = false;
            auto load = [&](int ch) {
                const int64_t q = q0 + (int64_t)ch * kCh + lane;
                rv = ch < nch && q < q1;
                if (rv) {
                    rx = a.x[q];
                    ry = a.y[q];
                    rh = a.h[q];
                    rw = a.w[q];
                }
            };
            const int c0 = (int)((sp - g) & 1u);
            if (c0 < nch) load(c0);
            for (int ch = c0; ch < nch; ch += 2) {
                const unsigned gc = g + ch;
                if (ch >= 2 && !tc::mbar_wait(tc::smem_addr(&bar_full[sp]), ((gc - 2) >> 1) & 1u, kWaitLimit))
                    atomicOr(a.status, ST_TIMEOUT);
                tc_prep_sample(ff, cc, rv, rx, ry, rh, rw, inv_cm, inv_nf, prep + sp * kPrepF * kCh, lane, a.status);
                if (ch + 2 < nch) load(ch + 2);
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_addr(&bar_prep[sp]));
            }
        } else {
            // ---- operand warps
            const int k = (lane & 7) + 8 * (warp & 3), o = (lane >> 3) + 4 * (warp >> 2);
            for (int ch = 0; ch < nch; ++ch) {
                const unsigned gc = g + ch, st = gc & 1u, use = gc >> 1;
                if (!tc::mbar_wait(tc::smem_addr(&bar_prep[st]), use & 1u, kWaitLimit)) atomicOr(a.status, ST_TIMEOUT);
                if (use > 0 && !tc::mbar_wait(tc::smem_addr(&bar_mma[st]), (use - 1) & 1u, kWaitLimit))
                    atomicOr(a.status, ST_TIMEOUT);
                if (ch >= 2 * kBlockChunks && ch % kBlockChunks == 0) {
                    // the run two blocks back is complete (the stage wait covers every earlier MMA):
                    // add it to the staged spectrum before its bank is reused
                    tc::fence_after_sync();
                    tc_flush(tmem + 128u * ((ch / kBlockChunks) & 1), hs, warp, lane);
                }
                const float* pr = prep + st * kPrepF * kCh;
                unsigned char* stg = smem + st * kStageBytes;
#pragma unroll
                for (int ax = 0; ax < 2; ++ax) {   // axis 0 -> A (y, times c), 1 -> B (x)
                    const float th = pr[(ax ? 1 : 3) * kCh + k], tl = pr[(ax ? 2 : 4) * kCh + k];
                    const float wr = pr[(ax ? 5 : 7) * kCh + k], wi = pr[(ax ? 6 : 8) * kCh + k];
                    float re[8], im[8];
                    tc_phasors<FULL>(th, tl, wr, wi, ax ? 1.0f : pr[k], 8 * o - half, 8 * o, P, re, im);
                    uint4 rh, rl, ih, il;
                    tc_split8(re, rh, rl);
                    tc_split8(im, ih, il);
                    unsigned char* hi = stg + (ax ? 2 : 0) * kOpBytes;
                    unsigned char* lo = hi + kOpBytes;
                    *reinterpret_cast<uint4*>(hi + tc::tc_off(8 * o, k)) = rh;
                    *reinterpret_cast<uint4*>(lo + tc::tc_off(8 * o, k)) = rl;
                    *reinterpret_cast<uint4*>(hi + tc::tc_off(64 + 8 * o, k)) = ih;
                    *reinterpret_cast<uint4*>(lo + tc::tc_off(64 + 8 * o, k)) = il;
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                tc::mbar_arrive(tc::smem_addr(&bar_full[st]));
            }
            // ---- the last one or two runs -> staged spectrum, scaled back by max |c|
            if (nch > 0) {
                const unsigned gl = g + nch - 1;
                if (!tc::mbar_wait(tc::smem_addr(&bar_mma[gl & 1u]), (gl >> 1) & 1u, kWaitLimit))
                    atomicOr(a.status, ST_TIMEOUT);
                tc::fence_after_sync();
                const int nb = (nch + kBlockChunks - 1) / kBlockChunks;
                for (int b = nb >= 2 ? nb - 2 : 0; b < nb; ++b) tc_flush(tmem + 128u * (b & 1), hs, warp, lane);
                for (int i = tid; i < 64 * kHS; i += kFeatThreads) hs[i] = cplx<float>{hs[i].re * cm, hs[i].im * cm};
            }
        }
        g += (unsigned)nch;
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        {
            float2* out = reinterpret_cast<float2*>(a.coeffs + (size_t)cell * P * P);
            for (int i = tid; i < P * P; i += kTcThreads) {
                const cplx<float> z = hs[(i / P) * kHS + (i % P)];
                out[i] = make_float2(z.re, z.im);
            }
        }
        if (a.do_ems) ems_rank_block<float, 8>(TcSpec{hs, half}, P, cell, a.ems, a.ems_out, ems_sm);
        __syncthreads();
    }
    // ---- every issued MMA has completed (each cell's operand warps waited for its last commit)
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// one block waiting on an mbarrier that never completes (no arrivals): the bounded wait gives up
static __global__ void tc_wait_timeout_kernel(unsigned polls, unsigned* status) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_addr(&bar), 1);
        tc::mbar_init_fence();
    }
    __syncthreads();
    if (!tc::mbar_wait(tc::smem_addr(&bar), 0u, polls) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

cudaError_t launch_wait_timeout(unsigned polls, unsigned* status, cudaStream_t s) {
    tc_wait_timeout_kernel<<<1, 32, 0, s>>>(polls, status);
    return cudaGetLastError();
}

cudaError_t tc_prepare() {
    cudaError_t e = cudaFuncSetAttribute(tc_nudft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_nudft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    return e;
}

cudaError_t launch_tc_nudft(const TcLaunch& l, cudaStream_t s) {
    if (l.n_list <= 0) return cudaSuccess;
    TcArgs a;
    a.x = l.x;
    a.y = l.y;
    a.h = l.h;
    a.w = l.w;
    a.offsets = l.offsets;
    a.cells = l.cells;
    a.list = l.list;
    a.n_list = l.n_list;
    a.P = l.P;
    a.NF = l.NF;
    a.coeffs = l.coeffs;
    a.status = l.status;
    a.do_ems = l.ems ? 1 : 0;
    if (l.ems) a.ems = *l.ems;
    else memset(&a.ems, 0, sizeof(a.ems));
    a.ems_out = l.ems_out;
    const int grid = l.n_list < 2 * l.num_sms ? l.n_list : 2 * l.num_sms;
    if (l.P == 64) tc_nudft_kernel<true><<<grid, kTcThreads, kSmemBytes, s>>>(a);
    else tc_nudft_kernel<false><<<grid, kTcThreads, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace enufft
