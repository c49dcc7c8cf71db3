// ems.cuh -- Elastic Mode Selection of one spectrum by one thread block (Sec. 2.2).
//
// Candidates are the mode pairs +-(m, n) of the symmetric box |m|, |n| <= P/2 - 1, named by the
// half-plane member (n > 0, or n == 0 and m > 0), p = (n + P/2) P + (m + P/2).  The block
//   1. forms every pair energy E_p = |h_p|^2 + |h_-p|^2 (times W_p), Eqs. energy / weighted_e,
//      with one fixed evaluation order so that reruns are bitwise identical;
//   2. selects the K_max largest by a segmented tournament: each warp ranks its own segment
//      (per-lane sorted registers, warp-wide argmax rounds), then one warp merges the sorted
//      warp lists (Eq. sorted_energy; ties go to the lower pair index);
//   3. evaluates N_eff, S_delta, C, alpha_C and the cumulative fraction theta(K) in binary64 and
//      thresholds it (Eqs. n_eff, s_delta, c_score, alpha_c, f_cum, k_elastic), in the same
//      operation order as the definition so that equal energies give equal decisions.
#pragma once

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

__device__ __forceinline__ bool key_better(const EmsKey& a, const EmsKey& b) {
    return a.e > b.e || (a.e == b.e && a.q > b.q);
}
__device__ __forceinline__ EmsKey key_shfl_xor(const EmsKey& k, int m) {
    EmsKey r;
    r.e = __shfl_xor_sync(0xffffffffu, k.e, m);
    r.q = __shfl_xor_sync(0xffffffffu, k.q, m);
    r.pad_ = 0;
    return r;
}
__device__ __forceinline__ bool key_is_pad(const EmsKey& k) { return k.e == 0ull && k.q == 0u; }

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
    static __device__ __forceinline__ double value(unsigned long long b) { return (double)__uint_as_float((unsigned)b); }
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
    static __device__ __forceinline__ double value(unsigned long long b) { return __longlong_as_double((long long)b); }
};

// shared-memory scratch of the block EMS: nwarps * k_max list keys + k_max merged keys + reductions
__host__ __device__ constexpr size_t ems_smem_bytes(int nwarps, int k_max) {
    return sizeof(EmsKey) * (size_t)(nwarps + 1) * k_max + sizeof(double) * 2 * nwarps + sizeof(int) * nwarps + 64;
}

// Block-wide EMS of one spectrum.  Spec provides get(m, n) -> cplx<T> for m, n in [-P/2, P/2).
// R: upper bound of candidates per lane per warp segment (compile time).  All threads of the
// block must call it; it ends with a __syncthreads().
template <typename T, int R, typename Spec>
__device__ void ems_block(const Spec& spec, int P, int cell, const EmsArgs& a, unsigned char* smem) {
    using EN = EnergyOf<T>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int half = P / 2, lim = half - 1, row = 2 * lim + 1;
    const int J = (lim > 0 ? lim + lim * row : 0) + (a.include_dc ? 1 : 0);
    const int K = a.k_max;
    EmsKey* lists = reinterpret_cast<EmsKey*>(smem);
    EmsKey* top = lists + (size_t)nwarps * K;
    double* red = reinterpret_cast<double*>(top + K);
    int* cnt = reinterpret_cast<int*>(red + 2 * nwarps);
    const double* Wc = a.W ? a.W + (a.w_per_cell ? (size_t)cell * P * P : 0) : nullptr;

    // ---- 1. energies of this warp's segment (register-major: slot r of lane l = r * 32 + l)
    const int seg = (J + nwarps - 1) / nwarps;
    const int s0 = warp * seg, s1 = min(J, s0 + seg);
    EmsKey key[R];
    double m1 = 0.0, m2 = 0.0;
    int npos = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = s0 + r * 32 + lane;
        key[r] = EmsKey{0ull, 0u, 0u};
        if (j < s1) {
            int m, n;
            bool dc = false;
            if (a.include_dc && j == J - 1) {
                m = 0; n = 0; dc = true;
            } else if (j < lim) {
                m = j + 1; n = 0;
            } else {
                const int jj = j - lim;
                n = 1 + jj / row;
                m = jj % row - lim;
            }
            const int p = (n + half) * P + (m + half);
            const T e = EN::pair(spec.get(m, n), spec.get(-m, -n), dc, Wc ? Wc[p] : 1.0, Wc != nullptr);
            key[r] = EmsKey{EN::bits(e), ~(unsigned)p, 0u};
            const double ed = (double)e;
            m1 += ed;
            m2 += ed * ed;
            npos += ed > 0.0;
        }
    }
    // per-lane descending order of the R slots (small sorting network)
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int k = R - 1; k > i; --k)
            if (key_better(key[k], key[k - 1])) {
                EmsKey t = key[k]; key[k] = key[k - 1]; key[k - 1] = t;
            }
    // ---- 2a. warp tournament: K rounds of a 32-way argmax over the lanes' heads
    int got = 0;
    for (int k = 0; k < K; ++k) {
        EmsKey best = key[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            EmsKey other = key_shfl_xor(best, o);
            if (key_better(other, best)) best = other;
        }
        if (key_is_pad(best)) break;
        const bool mine = (key[0].e == best.e && key[0].q == best.q);
        if (mine) {
#pragma unroll
            for (int r = 0; r < R - 1; ++r) key[r] = key[r + 1];
            key[R - 1] = EmsKey{0ull, 0u, 0u};
        }
        if (lane == 0) lists[(size_t)warp * K + k] = best;
        ++got;
    }
    // reductions for the ALL reading and for the positive count
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m1 += __shfl_xor_sync(0xffffffffu, m1, o);
        m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        npos += __shfl_xor_sync(0xffffffffu, npos, o);
    }
    if (lane == 0) {
        red[2 * warp] = m1;
        red[2 * warp + 1] = m2;
        cnt[warp] = got | (npos << 8);
    }
    __syncthreads();
    // ---- 2b. merge of the sorted warp lists by warp 0, then the scalar EMS by lane 0
    if (warp == 0) {
        int len = 0, pos = 0;
        EmsKey head{0ull, 0u, 0u};
        if (lane < nwarps) {
            len = cnt[lane] & 0xff;
            if (len > 0) head = lists[(size_t)lane * K];
        }
        int L = 0;
        for (int k = 0; k < K; ++k) {
            EmsKey best = head;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                EmsKey other = key_shfl_xor(best, o);
                if (key_better(other, best)) best = other;
            }
            if (key_is_pad(best)) break;
            if (lane < nwarps && head.e == best.e && head.q == best.q) {
                ++pos;
                head = pos < len ? lists[(size_t)lane * K + pos] : EmsKey{0ull, 0u, 0u};
            }
            if (lane == 0) top[k] = best;
            ++L;
        }
        __syncwarp();
        if (lane == 0) {
            int npos_all = 0;
            double A1 = 0.0, A2 = 0.0;
            for (int w = 0; w < nwarps; ++w) {
                npos_all += cnt[w] >> 8;
                A1 += red[2 * w];
                A2 += red[2 * w + 1];
            }
            const int Jmax = J < K ? J : K;
            double M1 = 0.0, M2 = 0.0;
            if (a.sum_over) {
                M1 = A1;
                M2 = A2;
            } else {
                for (int j = 0; j < Jmax; ++j) {
                    const double e = EN::value(top[j].e);
                    M1 = __dadd_rn(M1, e);
                    M2 = __dadd_rn(M2, __dmul_rn(e, e));
                }
            }
            const double neff = M2 > 0.0 ? __ddiv_rn(__dmul_rn(M1, M1), M2) : 0.0;
            double S = 0.0;
            if (Jmax >= 2) {
                for (int j = 0; j < Jmax - 1; ++j) {
                    const double e0 = EN::value(top[j].e), e1 = EN::value(top[j + 1].e);
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
                for (int j = 0; j < Jmax; ++j) {
                    cs = __dadd_rn(cs, EN::value(top[j].e));
                    if (cs >= __dmul_rn(alpha, total)) { kthr = j + 1; break; }
                }
                if (kthr < 0) kthr = K;
                Ks = kthr > a.k_min ? kthr : a.k_min;
                if (Ks > K) Ks = K;
                if (Ks > npos_all) Ks = npos_all;
                if (Ks > J) Ks = J;
                if (Ks > L) Ks = L;
                for (int j = 0; j < Ks; ++j) cum = __dadd_rn(cum, EN::value(top[j].e));
            }
            a.kstar[cell] = Ks;
            a.retained[cell] = cum;
            cnt[0] = Ks;
        }
        __syncwarp();
        const int Ks = cnt[0];
        for (int k = lane; k < K; k += 32)
            a.sel[(size_t)cell * K + k] = k < Ks ? (int)(~top[k].q) : -1;
    }
    __syncthreads();
}

}  // namespace enufft
