// autotune.cu -- plan-time tuning of the execution routes, and its on-disk cache.
//
// What is tuned (for mixed-precision plans whose cells take the fused or the tensor-core route):
//   - the routing threshold: the largest cell size, up to the caller's cap (opts.tc_max_points), at
//     which the tensor-core direct sum beats the fused spread/FFT kernel per sample;
//   - the persistent grid of the fused kernel: one or two resident blocks per SM.
// Both are measured on synthetic batches drawn from the plan's own cells: every synthetic cell
// copies the frame of one plan cell and holds Q samples spread uniformly over its window (rejection
// from the bounding box of the polygon), with a smooth elevation, for Q on a ladder of sizes.  Each
// candidate is timed with CUDA events on the plan's stream (one warm-up launch, the best of three).
//
// The cache is a JSON object {"key": {fields}, ...} in a file the caller names; a key holds the GPU
// name and SM count, P, n_f, w, precision, kernel, frame and the tensor-core cap, so a hit is only
// taken for an identical configuration on the same kind of GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "enufft.h"
#include "internal.h"

namespace enufft {

namespace {

constexpr int kTuneThreads = 256;

__device__ __forceinline__ unsigned tune_hash(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ double tune_unit(unsigned a, unsigned b) {
    return (double)(tune_hash(a * 0x9E3779B9U + tune_hash(b)) >> 8) * (1.0 / 16777216.0);
}

// synthetic cell i takes the frame of plan cell (i * stride) mod n_src
__global__ void tune_gather_cells(const CellConst* __restrict__ src, int n_src, int stride, CellConst* __restrict__ dst,
                                  int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[(int)(((int64_t)i * stride) % n_src)];
}

// Q samples per synthetic cell, uniform over the window of its frame (cell mask: rejection from the
// polygon's bounding box, up to 32 draws, the centroid as the last resort), elevation a smooth
// field of a few hundred metres, weight |D| / Q
// sample idx of a cell with Q samples: uniform over the cell's window (rejection from its bounding
// box with a counter-based hash), a smooth elevation, weights |D| / Q
__device__ __forceinline__ void tune_sample(const CellConst& cc, int64_t idx, int64_t Q, float* __restrict__ x,
                                            float* __restrict__ y, float* __restrict__ h, float* __restrict__ w,
                                            int64_t out) {
    double lox = -cc.H, hix = cc.H, loy = -cc.H, hiy = cc.H;
    if (cc.mask == 0 && cc.nv >= 3) {
        lox = hix = cc.ux[0];
        loy = hiy = cc.uy[0];
        for (int i = 1; i < cc.nv; ++i) {
            lox = fmin(lox, cc.ux[i]); hix = fmax(hix, cc.ux[i]);
            loy = fmin(loy, cc.uy[i]); hiy = fmax(hiy, cc.uy[i]);
        }
    }
    double ux = 0.0, uy = 0.0;
    for (unsigned t = 0; t < 32; ++t) {
        const double px = lox + (hix - lox) * tune_unit((unsigned)idx, 2 * t);
        const double py = loy + (hiy - loy) * tune_unit((unsigned)idx, 2 * t + 1);
        bool in = fabs(px) <= cc.H && fabs(py) <= cc.H;
        if (in && cc.mask == 2) in = px * px + py * py <= cc.H * cc.H;
        if (in && cc.mask == 0) {
            for (int i = 0; i < cc.nv && in; ++i) {
                const int j = (i + 1 == cc.nv) ? 0 : i + 1;
                const double cr = (cc.ux[j] - cc.ux[i]) * (py - cc.uy[i]) - (cc.uy[j] - cc.uy[i]) * (px - cc.ux[i]);
                in = cc.orient * cr >= 0.0;
            }
        }
        if (in) {
            ux = px;
            uy = py;
            break;
        }
    }
    x[out] = (float)(cc.cx + ux);
    y[out] = (float)(cc.cy + uy);
    h[out] = (float)(300.0 + 400.0 * sin(9.0 * ux / cc.H) * cos(7.0 * uy / cc.H));
    w[out] = (float)(cc.area / (double)Q);
}

__global__ void tune_samples(const CellConst* __restrict__ cells, int n, int Q, float* __restrict__ x,
                             float* __restrict__ y, float* __restrict__ h, float* __restrict__ w) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * Q) return;
    tune_sample(cells[idx / Q], idx, Q, x, y, h, w, idx);
}

// the same for cells with their own counts (offsets relative to p0), one block per cell
__global__ void tune_samples_off(const CellConst* __restrict__ cells, const int64_t* __restrict__ offsets, int64_t p0,
                                 float* __restrict__ x, float* __restrict__ y, float* __restrict__ h,
                                 float* __restrict__ w) {
    const int c = blockIdx.x;
    const int64_t q0 = offsets[c], q1 = offsets[c + 1];
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x)
        tune_sample(cells[c], q, q1 - q0, x, y, h, w, q - p0);
}

struct Dev {
    void* p = nullptr;
    ~Dev() {
        if (p) cudaFree(p);
    }
};

}  // namespace

cudaError_t autotune_run(const TuneEnv& env, enufft_tuning* out) {
    memset(out, 0, sizeof(*out));
    out->fused_blocks_per_sm = env.fwd_per_sm;
    out->tc_max_points = env.tc_cap;
    const int n = std::max(1, env.num_sms * std::max(1, env.fwd_per_sm) * 4);   // about four cells per block
    std::vector<int> ladder;
    if (env.tc_cap > 0)
        for (int q : {128, 256, 512, 1024, 2048, 3072, 4096, 6144})
            if (q <= env.tc_cap) ladder.push_back(q);
    const int q_grid = std::min(8192, std::max(256, env.q_median));
    const int q_max = std::max(q_grid, ladder.empty() ? 0 : ladder.back());
    Dev cells, x, y, h, w, off, order, co, ks, sel, ret, keys, info, ticket;
    cudaError_t e;
    const size_t np = (size_t)n * q_max;
    if ((e = cudaMalloc(&cells.p, sizeof(CellConst) * n)) != cudaSuccess ||
        (e = cudaMalloc(&x.p, 4 * np)) != cudaSuccess || (e = cudaMalloc(&y.p, 4 * np)) != cudaSuccess ||
        (e = cudaMalloc(&h.p, 4 * np)) != cudaSuccess || (e = cudaMalloc(&w.p, 4 * np)) != cudaSuccess ||
        (e = cudaMalloc(&off.p, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
        (e = cudaMalloc(&order.p, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMalloc(&co.p, sizeof(cplx<float>) * (size_t)n * env.P * env.P)) != cudaSuccess ||
        (e = cudaMalloc(&ks.p, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMalloc(&sel.p, sizeof(int) * n * kEmsMaxK)) != cudaSuccess ||
        (e = cudaMalloc(&ret.p, sizeof(double) * n)) != cudaSuccess ||
        (e = cudaMalloc(&keys.p, sizeof(EmsKey) * kEmsMaxK * n)) != cudaSuccess ||
        (e = cudaMalloc(&info.p, sizeof(EmsCellInfo) * n)) != cudaSuccess ||
        (e = cudaMalloc(&ticket.p, sizeof(unsigned))) != cudaSuccess)
        return e;
    const int stride = env.n_cells > 1 ? std::max(1, env.n_cells / n) : 1;
    tune_gather_cells<<<(n + 127) / 128, 128, 0, env.stream>>>(env.cells, std::max(1, env.n_cells), stride,
                                                              (CellConst*)cells.p, n);
    {
        std::vector<int> ord(n);
        for (int i = 0; i < n; ++i) ord[i] = i;
        if ((e = cudaMemcpyAsync(order.p, ord.data(), sizeof(int) * n, cudaMemcpyHostToDevice, env.stream)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(env.stream)) != cudaSuccess) return e;
    }
    EmsArgs ea;
    memset(&ea, 0, sizeof(ea));
    ea.k_min = 1;
    ea.k_max = 12;
    ea.alpha_max = 0.7;
    ea.delta = 0.02;
    ea.w1 = ea.w2 = 0.5;
    ea.kstar = (int32_t*)ks.p;
    ea.sel = (int32_t*)sel.p;
    ea.retained = (double*)ret.p;
    const EmsScratch sc{(EmsKey*)keys.p, (EmsCellInfo*)info.p};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto fill = [&](int Q) -> cudaError_t {
        std::vector<int64_t> o(n + 1);
        for (int i = 0; i <= n; ++i) o[i] = (int64_t)i * Q;
        cudaError_t r = cudaMemcpyAsync(off.p, o.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, env.stream);
        if (r != cudaSuccess) return r;
        const int64_t tot = (int64_t)n * Q;
        tune_samples<<<(unsigned)((tot + kTuneThreads - 1) / kTuneThreads), kTuneThreads, 0, env.stream>>>(
            (const CellConst*)cells.p, n, Q, (float*)x.p, (float*)y.p, (float*)h.p, (float*)w.p);
        r = cudaGetLastError();
        return r == cudaSuccess ? cudaStreamSynchronize(env.stream) : r;
    };
    auto best_of = [&](auto launch) -> double {   // ms, one warm-up then the best of three
        double best = 1e30;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, env.stream);
            if (launch() != cudaSuccess) return -1.0;
            cudaEventRecord(e1, env.stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, (double)ms);
        }
        return best;
    };
    FwdArgs<float> fa;
    memset(&fa, 0, sizeof(fa));
    fa.x = (const float*)x.p;
    fa.y = (const float*)y.p;
    fa.h = (const float*)h.p;
    fa.w = (const float*)w.p;
    fa.coeffs = (float*)co.p;
    fa.offsets = (const int64_t*)off.p;
    fa.cells = (const CellConst*)cells.p;
    fa.order = (const int*)order.p;
    fa.n_work = n;
    fa.P = env.P;
    fa.ticket = (unsigned*)ticket.p;
    fa.status = env.status;
    fa.twiddle = (const cplx<float>*)env.twiddle;
    for (int k = 0; k <= env.P / 2; ++k) fa.inv_phi[k] = (float)env.inv_phi[k];
    fa.poly = env.poly;
    fa.beta = env.beta;
    fa.do_ems = 1;
    fa.ems = ea;
    fa.ems_out = sc;
    auto fused = [&](int per_sm) {
        return [&, per_sm]() -> cudaError_t {
            cudaError_t r = cudaMemsetAsync(ticket.p, 0, sizeof(unsigned), env.stream);
            if (r != cudaSuccess) return r;
            return launch_type1(fa, env.NF, env.W, std::min(n, per_sm * env.num_sms), env.stream);
        };
    };
    TcLaunch tl;
    memset(&tl, 0, sizeof(tl));
    tl.x = fa.x;
    tl.y = fa.y;
    tl.h = fa.h;
    tl.w = fa.w;
    tl.offsets = fa.offsets;
    tl.cells = fa.cells;
    tl.list = (const int*)order.p;
    tl.n_list = n;
    tl.P = env.P;
    tl.NF = env.NF;
    tl.num_sms = env.num_sms;
    tl.coeffs = (cplx<float>*)co.p;
    tl.status = env.status;
    tl.ems = &ea;
    tl.ems_out = sc;
    auto tc = [&]() -> cudaError_t { return launch_tc_nudft(tl, env.stream); };

    // the fused kernel's grid at the plan's typical cell size
    if ((e = fill(q_grid)) != cudaSuccess) return e;
    if (env.fwd_per_sm > 1) {
        const double t1 = best_of(fused(1)), t2 = best_of(fused(env.fwd_per_sm));
        if (t1 < 0 || t2 < 0) return cudaGetLastError();
        out->fused_blocks_per_sm = t1 < t2 ? 1 : env.fwd_per_sm;
    }
    // the routing threshold: the largest size of the ladder at which the direct sum is faster
    out->tc_max_points = 0;
    out->n_ladder = (int)ladder.size();
    for (size_t i = 0; i < ladder.size(); ++i) {
        const int Q = ladder[i];
        if ((e = fill(Q)) != cudaSuccess) return e;
        const double tf = best_of(fused(out->fused_blocks_per_sm)), tt = best_of(tc);
        if (tf < 0 || tt < 0) return cudaGetLastError();
        out->ladder[i] = Q;
        out->ns_fused[i] = 1e6 * tf / ((double)n * Q);
        out->ns_tc[i] = 1e6 * tt / ((double)n * Q);
        if (out->ns_tc[i] < out->ns_fused[i]) out->tc_max_points = Q;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cudaStreamSynchronize(env.stream);
}

// ---------------------------------------------------------------------------------------------
// cache file
// ---------------------------------------------------------------------------------------------
namespace {

// the objects of a file {"key": {...}, ...} by key; false if the text is not of that form
bool parse_cache(const std::string& s, std::map<std::string, std::string>& out) {
    size_t i = 0;
    auto ws = [&]() {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\t' || s[i] == '\r')) ++i;
    };
    ws();
    if (i >= s.size() || s[i] != '{') return false;
    ++i;
    ws();
    if (i < s.size() && s[i] == '}') return true;
    for (;;) {
        ws();
        if (i >= s.size() || s[i] != '"') return false;
        const size_t k0 = ++i;
        while (i < s.size() && s[i] != '"') ++i;
        if (i >= s.size()) return false;
        const std::string key = s.substr(k0, i - k0);
        ++i;
        ws();
        if (i >= s.size() || s[i] != ':') return false;
        ++i;
        ws();
        if (i >= s.size() || s[i] != '{') return false;
        const size_t v0 = i;
        int depth = 0;
        for (; i < s.size(); ++i) {
            if (s[i] == '{') ++depth;
            if (s[i] == '}' && --depth == 0) break;
        }
        if (i >= s.size()) return false;
        out[key] = s.substr(v0, i - v0 + 1);
        ++i;
        ws();
        if (i < s.size() && s[i] == ',') {
            ++i;
            continue;
        }
        return i < s.size() && s[i] == '}';
    }
}

bool field_num(const std::string& obj, const char* name, double& v) {
    const std::string pat = std::string("\"") + name + "\"";
    const size_t p = obj.find(pat);
    if (p == std::string::npos) return false;
    const size_t c = obj.find(':', p + pat.size());
    if (c == std::string::npos) return false;
    char* end = nullptr;
    v = strtod(obj.c_str() + c + 1, &end);
    return end != obj.c_str() + c + 1;
}

int field_arr(const std::string& obj, const char* name, double* v, int cap) {
    const std::string pat = std::string("\"") + name + "\"";
    const size_t p = obj.find(pat);
    if (p == std::string::npos) return -1;
    size_t i = obj.find('[', p + pat.size());
    const size_t j = obj.find(']', p + pat.size());
    if (i == std::string::npos || j == std::string::npos || j < i) return -1;
    int k = 0;
    ++i;
    while (i < j && k < cap) {
        char* end = nullptr;
        const double d = strtod(obj.c_str() + i, &end);
        if (end == obj.c_str() + i) break;
        v[k++] = d;
        i = (size_t)(end - obj.c_str());
        while (i < j && (obj[i] == ',' || obj[i] == ' ')) ++i;
    }
    return k;
}

std::string tuning_json(const enufft_tuning& t) {
    std::string s = "{\"tc_max_points\": " + std::to_string(t.tc_max_points) +
                    ", \"fused_blocks_per_sm\": " + std::to_string(t.fused_blocks_per_sm) +
                    ", \"large_tile\": " + std::to_string(t.large_tile) + ", \"ladder\": [";
    char buf[64];
    for (int i = 0; i < t.n_ladder; ++i) s += (i ? ", " : "") + std::to_string(t.ladder[i]);
    s += "], \"ns_fused\": [";
    for (int i = 0; i < t.n_ladder; ++i) {
        snprintf(buf, sizeof buf, "%s%.6g", i ? ", " : "", t.ns_fused[i]);
        s += buf;
    }
    s += "], \"ns_tc\": [";
    for (int i = 0; i < t.n_ladder; ++i) {
        snprintf(buf, sizeof buf, "%s%.6g", i ? ", " : "", t.ns_tc[i]);
        s += buf;
    }
    return s + "]}";
}

bool read_file(const char* path, std::string& s) {
    FILE* f = fopen(path, "rb");
    if (!f) return false;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, r);
    fclose(f);
    return true;
}

}  // namespace

cudaError_t large_tune_samples(const CellConst* cells, const int64_t* offsets, int64_t p0, int ncells, float* x,
                               float* y, float* h, float* w, cudaStream_t s) {
    if (ncells <= 0) return cudaSuccess;
    tune_samples_off<<<ncells, kTuneThreads, 0, s>>>(cells, offsets, p0, x, y, h, w);
    return cudaGetLastError();
}

bool tune_cache_get(const char* path, const std::string& key, enufft_tuning* out) {
    std::string s;
    std::map<std::string, std::string> m;
    if (!path || !read_file(path, s) || !parse_cache(s, m)) return false;
    const auto it = m.find(key);
    if (it == m.end()) return false;
    enufft_tuning t;
    memset(&t, 0, sizeof(t));
    double v;
    if (!field_num(it->second, "tc_max_points", v)) return false;
    t.tc_max_points = (int)v;
    if (!field_num(it->second, "fused_blocks_per_sm", v)) return false;
    t.fused_blocks_per_sm = (int)v;
    double a[8];
    const int nl = field_arr(it->second, "ladder", a, 8);
    if (nl < 0) return false;
    t.n_ladder = nl;
    for (int i = 0; i < nl; ++i) t.ladder[i] = (int)a[i];
    if (field_arr(it->second, "ns_fused", t.ns_fused, 8) != nl || field_arr(it->second, "ns_tc", t.ns_tc, 8) != nl)
        return false;
    t.large_tile = field_num(it->second, "large_tile", v) ? (int)v : 0;   // older records: none
    if (t.tc_max_points < 0 || t.fused_blocks_per_sm < 1) return false;
    t.from_cache = 1;
    *out = t;
    return true;
}

bool tune_cache_put(const char* path, const std::string& key, const enufft_tuning& t) {
    if (!path) return false;
    std::string s;
    std::map<std::string, std::string> m;
    if (read_file(path, s) && !parse_cache(s, m)) m.clear();   // an unreadable cache is replaced
    m[key] = tuning_json(t);
    std::string o = "{\n";
    bool first = true;
    for (const auto& kv : m) {
        o += (first ? "  \"" : ",\n  \"") + kv.first + "\": " + kv.second;
        first = false;
    }
    o += "\n}\n";
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return false;
    const bool ok = fwrite(o.data(), 1, o.size(), f) == o.size();
    fclose(f);
    return ok && rename(tmp.c_str(), path) == 0;
}

}  // namespace enufft

extern "C" enufft_status enufft_tune_cache_lookup(const char* path, const char* key, enufft_tuning* out) {
    if (!path || !key || !out) {
        enufft::set_thread_error("tune_cache_lookup: NULL argument");
        return ENUFFT_ERR_ARG;
    }
    if (!enufft::tune_cache_get(path, key, out)) {
        enufft::set_thread_error("tune_cache_lookup: no entry for the key (or the file is missing or malformed)");
        return ENUFFT_ERR_ARG;
    }
    return ENUFFT_OK;
}

extern "C" enufft_status enufft_tune_cache_store(const char* path, const char* key, const enufft_tuning* t) {
    if (!path || !key || !t || strchr(key, '"') || strchr(key, '\\')) {
        enufft::set_thread_error("tune_cache_store: NULL argument or a key with a quote or backslash");
        return ENUFFT_ERR_ARG;
    }
    if (t->n_ladder < 0 || t->n_ladder > 8 || t->tc_max_points < 0 || t->fused_blocks_per_sm < 1) {
        enufft::set_thread_error("tune_cache_store: tuning record out of range");
        return ENUFFT_ERR_ARG;
    }
    if (!enufft::tune_cache_put(path, key, *t)) {
        enufft::set_thread_error("tune_cache_store: cannot write the cache file");
        return ENUFFT_ERR_ARG;
    }
    return ENUFFT_OK;
}
