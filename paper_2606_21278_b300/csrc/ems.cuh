// ems.cuh -- Elastic Mode Selection (Sec. 2.2) in two stages.
//
// Candidates are the mode pairs +-(m, n) of the symmetric box |m|, |n| <= P/2 - 1, named by the
// half-plane member (n > 0, or n == 0 and m > 0), p = (n + P/2) P + (m + P/2).
//
// Stage 1, ranking (one thread block per spectrum, inside the fused transform kernel or the
// standalone EMS kernel):
//   - every pair energy E_p = |h_p|^2 + |h_-p|^2 (times W_p), Eqs. energy / weighted_e, formed in
//     one fixed evaluation order so that reruns are bitwise identical;
//   - the K_max largest (Eq. sorted_energy; ties go to the lower pair index) by a radix select on
//     the energy bits followed by a small ordering of the survivors;
//   - the number of positive energies and, for the ALL reading only, sum E and sum E^2 over all
//     pairs as unevaluated binary32 pairs (error-free transformations, ~48-bit accurate);
//   written to per-cell scratch.
// Stage 2, the elastic count (one thread per cell, binary64): N_eff, S_delta, C, alpha_C, the
// cumulative fraction theta(K) and K* (Eqs. n_eff, s_delta, c_score, alpha_c, f_cum, k_elastic),
// in the definition's operation order so that equal energies give equal decisions.  Doing this
// scalar binary64 work one cell per lane keeps B300's narrow binary64 pipe fully occupied instead
// of stalling a whole thread block on one lane.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace enufft {

constexpr int kEmsMaxK = 64;

struct EmsArgs {
    int k_min, k_max;
    double alpha_min, alpha_max, delta, w1, w2;
    int sum_over;      // 0 HEAD (J_max), 1 ALL (J*)
    int include_dc;
    const double* W;   // NULL, [P][P] or [n_cells][P][P]
    int w_per_cell;
    int32_t* kstar;
    int32_t* sel;
    double* retained;
};

// ranking key: energy bits (non-negative binary32 or binary64, so integer order = value order)
// and the complemented pair index (so that the lower index wins a tie)
struct EmsKey {
    unsigned long long e;
    unsigned int q;
    unsigned int pad_;
};

// per-cell result of stage 1
struct EmsCellInfo {
    int L;          // keys found (<= K_max)
    int J;          // candidate pairs J*
    int npos;       // pairs with positive energy
    int is_f64;     // energies are binary64 bits (else binary32 bits)
    float m1h, m1l, m2h, m2l;   // ALL reading: sum E and sum E^2 as hi + lo
    double m1d, m2d;            // ALL reading, binary64 energies
};

struct EmsScratch {
    EmsKey* keys;        // [n_cells][kEmsMaxK]
    EmsCellInfo* info;   // [n_cells]
};

__device__ __forceinline__ bool key_better(const EmsKey& a, const EmsKey& b) {
    return a.e > b.e || (a.e == b.e && a.q > b.q);
}

// error-free binary32 sum (Knuth TwoSum) and product (FMA)
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (ah + al) + (bh + bl) as a renormalised pair
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
    float s, e;
    two_sum_f(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    ah = __fadd_rn(s, e);
    al = __fsub_rn(e, __fsub_rn(ah, s));
}

// energy of the pair (m, n) in the kernel's fixed order; T = float -> binary32, double -> binary64
template <typename T>
struct EnergyOf;
template <>
struct EnergyOf<float> {
    static __device__ __forceinline__ float pair(cplx<float> a, cplx<float> b, bool dc, double W, bool hasW) {
        float ep = __fmaf_rn(a.re, a.re, __fmul_rn(a.im, a.im));
        float e = ep;
        if (!dc) e = __fadd_rn(ep, __fmaf_rn(b.re, b.re, __fmul_rn(b.im, b.im)));
        if (hasW) e = __fmul_rn(e, (float)W);
        return e;
    }
    static __device__ __forceinline__ unsigned long long bits(float e) { return (unsigned long long)__float_as_uint(e); }
};
template <>
struct EnergyOf<double> {
    static __device__ __forceinline__ double pair(cplx<double> a, cplx<double> b, bool dc, double W, bool hasW) {
        double e = __dadd_rn(__dmul_rn(a.re, a.re), __dmul_rn(a.im, a.im));
        if (!dc) e = __dadd_rn(e, __dadd_rn(__dmul_rn(b.re, b.re), __dmul_rn(b.im, b.im)));
        if (hasW) e = __dmul_rn(e, W);
        return e;
    }
    static __device__ __forceinline__ unsigned long long bits(double e) { return (unsigned long long)__double_as_longlong(e); }
};

__device__ __forceinline__ double key_value(const EmsKey& k, int is_f64) {
    return is_f64 ? __longlong_as_double((long long)k.e) : (double)__uint_as_float((unsigned)k.e);
}

// shared-memory scratch of stage 1: digit histogram, surviving keys, reductions
__host__ __device__ constexpr size_t ems_smem_bytes(int nwarps, int k_max) {
    return sizeof(unsigned) * 256 + sizeof(EmsKey) * (size_t)(k_max > 64 ? k_max : 64) + sizeof(float) * 4 * nwarps +
           sizeof(double) * 2 * nwarps + sizeof(int) * (2 * nwarps + 8) + 64;
}

// candidate j (0 .. J-1) -> mode (m, n); with the DC mode first when it is a candidate, the pair
// index p = (n + P/2) P + (m + P/2) increases with j, so "lower index first" is "lower j first"
__device__ __forceinline__ void ems_mode_of(int j, int lim, int row, int dc_first, int& m, int& n) {
    if (dc_first) {
        if (j == 0) { m = 0; n = 0; return; }
        --j;
    }
    if (j < lim) {
        m = j + 1;
        n = 0;
    } else {
        const int jj = j - lim;
        n = 1 + jj / row;
        m = jj % row - lim;
    }
}

// Stage 1 for one spectrum by the whole block.  Spec provides get(m, n) -> cplx<T> for
// m, n in [-P/2, P/2).  R: upper bound of candidates per thread (compile time).  All threads of
// the block must call it; it ends with a __syncthreads().
//
// The K_max largest energies are found by a most-significant-digit radix select on the energy
// bits (8-bit digits, one shared-memory histogram pass per digit).  As soon as the keys at or
// above the current digit prefix number at most kEmsCand, they are all kept and one warp ranks
// them exactly by (energy desc, index asc); otherwise the select runs to the last digit, which
// yields the K-th largest value T, and of the keys equal to T those with the lowest pair index
// are kept (block prefix count in candidate order).
constexpr int kEmsCand = 64;

template <typename T, int R, typename Spec>
__device__ void ems_rank_block(const Spec& spec, int P, int cell, const EmsArgs& a, const EmsScratch& out,
                               unsigned char* smem) {
    using EN = EnergyOf<T>;
    using U = typename std::conditional<sizeof(T) == 4, unsigned, unsigned long long>::type;
    constexpr int NDIG = (int)sizeof(U);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x, nwarps = nt >> 5;
    const int half = P / 2, lim = half - 1, row = 2 * lim + 1;
    const int dc = a.include_dc ? 1 : 0;
    const int J = (lim > 0 ? lim + lim * row : 0) + dc;
    const int K = a.k_max;
    unsigned* hist = reinterpret_cast<unsigned*>(smem);
    EmsKey* keep = reinterpret_cast<EmsKey*>(hist + 256);     // kEmsCand entries
    float* redf = reinterpret_cast<float*>(keep + kEmsCand);
    double* redd = reinterpret_cast<double*>(redf + 4 * nwarps);
    int* wsum = reinterpret_cast<int*>(redd + 2 * nwarps);     // [2 * nwarps]
    int* ctl = wsum + 2 * nwarps;                             // [0] digit, [2] remaining, [3] kept, [4] stop
    const double* Wc = a.W ? a.W + (a.w_per_cell ? (size_t)cell * P * P : 0) : nullptr;
    const bool all = a.sum_over != 0;

    // ---- energies, candidates j = tid * R + r (contiguous per thread, modes walked without division)
    U u[R];
    int pj[R];
    float m1h = 0.f, m1l = 0.f, m2h = 0.f, m2l = 0.f;
    double m1d = 0.0, m2d = 0.0;
    int npos = 0;
    {
        int m = 0, n = 0;
        const int j0 = tid * R;
        if (j0 < J) ems_mode_of(j0, lim, row, dc, m, n);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = j0 + r;
            u[r] = 0;
            pj[r] = 0;
            if (j < J) {
                const bool isdc = (m == 0 && n == 0);
                const int p = (n + half) * P + (m + half);
                const T e = EN::pair(spec.get(m, n), spec.get(-m, -n), isdc, Wc ? Wc[p] : 1.0, Wc != nullptr);
                u[r] = (U)EN::bits(e);
                pj[r] = p;
                npos += e > T(0);
                if (all) {
                    if constexpr (sizeof(T) == 4) {
                        const float sq = __fmul_rn(e, e), sqe = __fmaf_rn(e, e, -sq);
                        df_add(m1h, m1l, e, 0.f);
                        df_add(m2h, m2l, sq, sqe);
                    } else {
                        m1d += e;
                        m2d += e * e;
                    }
                }
                // next candidate in enumeration order
                if (isdc) {
                    m = 1; n = 0;
                } else if (++m > lim) {
                    m = -lim; ++n;
                }
            }
        }
    }
    const int Kt = K < J ? K : J;   // keys to keep
    // ---- radix select (digits from the most significant), with early exit
    U prefix = 0, pmask = 0;
    int remaining = Kt, stop = 0;
    if (tid == 0) ctl[3] = 0;
    for (int d = NDIG - 1; d >= 0 && Kt > 0; --d) {
        const int shift = 8 * d;
        for (int i = tid; i < 256; i += nt) hist[i] = 0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (tid * R + r < J && (u[r] & pmask) == prefix) atomicAdd(&hist[(unsigned)(u[r] >> shift) & 255u], 1u);
        __syncthreads();
        if (warp == 0) {
            // lane l owns digits 255 - 8l .. 248 - 8l (descending); exclusive scan from the top
            unsigned c8[8], tot = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) { c8[k] = hist[255 - 8 * lane - k]; tot += c8[k]; }
            unsigned incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            unsigned before = incl - tot;   // keys with a larger digit than this lane's first digit
            int found = -1;
            unsigned above = 0, inbin = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (found < 0 && before + c8[k] >= (unsigned)remaining && before < (unsigned)remaining) {
                    found = 255 - 8 * lane - k;
                    above = before;
                    inbin = c8[k];
                }
                before += c8[k];
            }
            const unsigned ball = __ballot_sync(0xffffffffu, found >= 0);
            const int src = __ffs(ball) - 1;
            const int dig = __shfl_sync(0xffffffffu, found, src);
            const unsigned ab = __shfl_sync(0xffffffffu, above, src);
            const unsigned ib = __shfl_sync(0xffffffffu, inbin, src);
            if (lane == 0) {
                ctl[0] = dig;
                ctl[2] = remaining - (int)ab;
                // keys already above (Kt - remaining) + this pass's keys above and in the digit
                ctl[4] = (Kt - remaining) + (int)(ab + ib) <= kEmsCand;
            }
        }
        __syncthreads();
        prefix |= (U)ctl[0] << shift;
        pmask |= (U)255 << shift;
        remaining = ctl[2];
        stop = ctl[4];
        __syncthreads();
        if (stop) break;
    }
    // ---- keep: everything at or above the prefix (early exit), or above T plus the first
    // `remaining` keys equal to T in candidate order (full depth)
    if (stop) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (tid * R + r < J && (u[r] & pmask) >= prefix) {
                const int slot = atomicAdd(&ctl[3], 1);
                keep[slot] = EmsKey{(unsigned long long)u[r], ~(unsigned)pj[r], 0u};
            }
        }
    } else if (Kt > 0) {
        int eq = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) eq += (tid * R + r < J && u[r] == prefix);
        int incl = eq;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int rank = incl - eq;   // equal keys before this thread, in candidate order
        for (int w = 0; w < warp; ++w) rank += wsum[w];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (tid * R + r < J) {
                bool take = u[r] > prefix;
                if (u[r] == prefix) take = rank++ < remaining;
                if (take) {
                    const int slot = atomicAdd(&ctl[3], 1);
                    keep[slot] = EmsKey{(unsigned long long)u[r], ~(unsigned)pj[r], 0u};
                }
            }
        }
    }
    // ---- reductions (positive count; ALL-reading sums)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npos += __shfl_xor_sync(0xffffffffu, npos, o);
    if (all) {
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float a1 = __shfl_xor_sync(0xffffffffu, m1h, o), b1 = __shfl_xor_sync(0xffffffffu, m1l, o);
                const float a2 = __shfl_xor_sync(0xffffffffu, m2h, o), b2 = __shfl_xor_sync(0xffffffffu, m2l, o);
                df_add(m1h, m1l, a1, b1);
                df_add(m2h, m2l, a2, b2);
            }
        } else {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                m1d += __shfl_xor_sync(0xffffffffu, m1d, o);
                m2d += __shfl_xor_sync(0xffffffffu, m2d, o);
            }
        }
    }
    __syncthreads();   // keep[] complete, wsum reads done
    if (lane == 0) {
        redf[4 * warp + 0] = m1h; redf[4 * warp + 1] = m1l;
        redf[4 * warp + 2] = m2h; redf[4 * warp + 3] = m2l;
        redd[2 * warp] = m1d; redd[2 * warp + 1] = m2d;
        wsum[nwarps + warp] = npos;
    }
    __syncthreads();
    // ---- rank the survivors over the whole block: thread t compares candidate t / 8 with the
    // eighth (t % 8) of the others, eight lanes sum the partial ranks; keep the first Kt
    {
        const int C = ctl[3];
        EmsKey* dst = out.keys + (size_t)cell * kEmsMaxK;
        const int i = tid >> 3, part = tid & 7;
        int rk = 0;
        EmsKey ki{0ull, 0u, 0u};
        if (i < C) {
            ki = keep[i];
            for (int k = part; k < C; k += 8) rk += key_better(keep[k], ki);
        }
        rk += __shfl_xor_sync(0xffffffffu, rk, 1);
        rk += __shfl_xor_sync(0xffffffffu, rk, 2);
        rk += __shfl_xor_sync(0xffffffffu, rk, 4);
        if (i < C && part == 0 && rk < Kt) dst[rk] = ki;
        // blocks narrower than 512 threads: further rounds (uniform trip count, so every lane
        // takes part in the shuffles)
        for (int base = nt / 8; base < C; base += nt / 8) {
            const int ii = base + i;
            EmsKey kj{0ull, 0u, 0u};
            int r2 = 0;
            if (ii < C) {
                kj = keep[ii];
                for (int k = part; k < C; k += 8) r2 += key_better(keep[k], kj);
            }
            r2 += __shfl_xor_sync(0xffffffffu, r2, 1);
            r2 += __shfl_xor_sync(0xffffffffu, r2, 2);
            r2 += __shfl_xor_sync(0xffffffffu, r2, 4);
            if (ii < C && part == 0 && r2 < Kt) dst[r2] = kj;
        }
    }
    if (warp == 0) {
        const int C = ctl[3];
        if (lane == 0) {
            EmsCellInfo inf;
            inf.L = C < Kt ? C : Kt;
            inf.J = J;
            inf.is_f64 = sizeof(T) == 8;
            int np = 0;
            float a1h = 0.f, a1l = 0.f, a2h = 0.f, a2l = 0.f;
            double d1 = 0.0, d2 = 0.0;
            for (int w = 0; w < nwarps; ++w) {
                np += wsum[nwarps + w];
                if (all) {
                    df_add(a1h, a1l, redf[4 * w], redf[4 * w + 1]);
                    df_add(a2h, a2l, redf[4 * w + 2], redf[4 * w + 3]);
                    d1 += redd[2 * w];
                    d2 += redd[2 * w + 1];
                }
            }
            inf.npos = np;
            inf.m1h = a1h; inf.m1l = a1l; inf.m2h = a2h; inf.m2l = a2l;
            inf.m1d = d1; inf.m2d = d2;
            out.info[cell] = inf;
        }
    }
    __syncthreads();
}

// Stage 2: one thread per cell, binary64, the definition's operation order.
static __global__ void ems_finish_kernel(int64_t n_cells, const __grid_constant__ EmsArgs a, EmsScratch s) {
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= n_cells) return;
    const EmsCellInfo inf = s.info[cell];
    const EmsKey* top = s.keys + (size_t)cell * kEmsMaxK;
    const int K = a.k_max, J = inf.J, L = inf.L, f64 = inf.is_f64;
    const int Jmax = J < K ? J : K;
    double M1 = 0.0, M2 = 0.0;
    if (a.sum_over) {
        if (f64) {
            M1 = inf.m1d;
            M2 = inf.m2d;
        } else {
            M1 = (double)inf.m1h + (double)inf.m1l;
            M2 = (double)inf.m2h + (double)inf.m2l;
        }
    } else {
        for (int j = 0; j < Jmax && j < L; ++j) {
            const double e = key_value(top[j], f64);
            M1 = __dadd_rn(M1, e);
            M2 = __dadd_rn(M2, __dmul_rn(e, e));
        }
    }
    const double neff = M2 > 0.0 ? __ddiv_rn(__dmul_rn(M1, M1), M2) : 0.0;
    double S = 0.0;
    if (Jmax >= 2) {
        for (int j = 0; j < Jmax - 1 && j + 1 < L; ++j) {
            const double e0 = key_value(top[j], f64), e1 = key_value(top[j + 1], f64);
            if (e1 > 0.0) S = __dadd_rn(S, exp(__ddiv_rn(-__dsub_rn(__ddiv_rn(e0, e1), 1.0), a.delta)));
        }
        S = __ddiv_rn(S, (double)(Jmax - 1));
    }
    const double nclip = neff < (double)K ? neff : (double)K;
    const double C = __dadd_rn(__ddiv_rn(__dmul_rn(a.w1, nclip), (double)K), __dmul_rn(a.w2, S));
    const double alpha = __dadd_rn(a.alpha_min, __dmul_rn(__dsub_rn(a.alpha_max, a.alpha_min), C));
    const double total = M1;
    int Ks = 0;
    double cum = 0.0;
    if (total > 0.0) {
        int kthr = -1;
        double cs = 0.0;
        for (int j = 0; j < Jmax && j < L; ++j) {
            cs = __dadd_rn(cs, key_value(top[j], f64));
            if (cs >= __dmul_rn(alpha, total)) { kthr = j + 1; break; }
        }
        if (kthr < 0) kthr = K;
        Ks = kthr > a.k_min ? kthr : a.k_min;
        if (Ks > K) Ks = K;
        if (Ks > inf.npos) Ks = inf.npos;
        if (Ks > J) Ks = J;
        if (Ks > L) Ks = L;
        for (int j = 0; j < Ks; ++j) cum = __dadd_rn(cum, key_value(top[j], f64));
    }
    a.kstar[cell] = Ks;
    a.retained[cell] = cum;
    int32_t* sel = a.sel + (size_t)cell * K;
    for (int k = 0; k < K; ++k) sel[k] = k < Ks ? (int)(~top[k].q) : -1;
}

}  // namespace enufft
