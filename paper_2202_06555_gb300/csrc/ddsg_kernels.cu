// ddsg_kernels.cu -- CUDA kernels of libddsg (sm_103a).
//
//   encode_queries   physical FP64 query -> clamped canonical fixed point (Sec. 2.2
//                    canonical domain), one warp per query.
//   eval_lq          DDSG interpolation (Sec. 4.1, eq. 4.2 / slice-free form):
//                    one thread per query, a chunk of MC outputs per thread,
//                    all components in one pass.
//   hierarchize      surpluses layer by layer (Sec. 3.1), one block per component.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "ddsg_internal.h"

namespace ddsg {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ double pow2m_d(int e) {  // 2^-e, 0 <= e < 1022
    return __longlong_as_double((long long)(1023 - e) << 52);
}
__device__ __forceinline__ float pow2m_f(int e) {  // 2^-e, 0 <= e < 126
    return __int_as_float((127 - e) << 23);
}

// ---------------------------------------------------------------------------
// query encoding
// ---------------------------------------------------------------------------

// One warp per query row: X[q*d + j] = fixed point of clamp((x - lo_j) / span_j).
// flags (n int32, stored after X) = 1 when any coordinate is non-finite.
// stats[0] += clamped coordinates, stats[1] += non-finite rows.
__global__ void __launch_bounds__(256) encode_queries_kernel(int64_t n, int d, const double *__restrict__ x,
                                                             const double *__restrict__ lo,
                                                             const double *__restrict__ span,
                                                             uint64_t *__restrict__ X,
                                                             int32_t *__restrict__ flags,
                                                             unsigned long long *__restrict__ stats) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long clamps = 0, nans = 0;
    for (int64_t q = warp; q < n; q += nwarps) {
        bool bad = false;
        for (int j = lane; j < d; j += 32) {
            const double xv = x[q * d + j];
            double c = (xv - lo[j]) / span[j];
            uint64_t Xv;
            if (!(c == c) || c == __longlong_as_double(0x7ff0000000000000ll) ||
                c == __longlong_as_double(0xfff0000000000000ll) || !(xv - xv == 0.0)) {
                bad = true;
                Xv = X_NAN;
            } else {
                if (c < 0.0) { c = 0.0; ++clamps; }
                if (c > 1.0) { c = 1.0; ++clamps; }
                const double yv = c * 4611686018427387904.0;  // c * 2^62, exact
                Xv = (uint64_t)yv;                              // floor (yv >= 0)
                if ((double)Xv != yv) Xv |= 1ull;               // sticky: strictly inside a cell
            }
            X[q * d + j] = Xv;
        }
        const bool any_bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            flags[q] = any_bad ? 1 : 0;
            if (any_bad) ++nans;
        }
    }
    // warp-level reduction of counters, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) clamps += __shfl_down_sync(0xffffffffu, clamps, o);
    if (lane == 0 && (clamps | nans)) {
        atomicAdd(&stats[0], clamps);
        atomicAdd(&stats[1], nans);
    }
}

cudaError_t launch_encode_queries(int64_t n, int d, const double *x, const double *lo,
                                  const double *span, uint64_t *X, int64_t *stats,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int32_t *flags = reinterpret_cast<int32_t *>(X + n * (int64_t)d);
    int64_t blocks = (n + 7) / 8;
    if (blocks > 152 * 64) blocks = 152 * 64;
    encode_queries_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, d, x, lo, span, X, flags,
                                                           reinterpret_cast<unsigned long long *>(stats));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// evaluation: lanes over queries
// ---------------------------------------------------------------------------

struct EvalParams {
    DevTables t;
    int d, m;
    int64_t n;
    const uint64_t *X;
    const int32_t *flags;
    double *y;
    uint64_t *hash;
    int32_t *count;
    int form;
};

// Accumulators: FP64 plain sums, or FP32 with Kahan compensation per term.
template <int PREC>
struct Acc;

template <>
struct Acc<DDSG_F64> {
    double s = 0.0;
    __device__ __forceinline__ void add(double w, double a) { s = fma(w, a, s); }
    __device__ __forceinline__ double result() const { return s; }
};

template <>
struct Acc<DDSG_F32C> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float w, float a) {
        const float term = __fmul_rn(w, a);
        const float yk = __fsub_rn(term, c);
        const float tk = __fadd_rn(s, yk);
        c = __fsub_rn(__fsub_rn(tk, s), yk);
        s = tk;
    }
    __device__ __forceinline__ double result() const { return (double)s - (double)c; }
};

template <int PREC, int MC, bool HC>
__global__ void __launch_bounds__(128) eval_lq_kernel(const EvalParams p) {
    using W = typename std::conditional<PREC == DDSG_F64, double, float>::type;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= p.n) return;
    const int m0 = blockIdx.y * MC;
    const int m = p.m;
    if (p.flags[q]) {
        for (int o = 0; o < MC; ++o)
            if (m0 + o < m) p.y[q * m + m0 + o] = __longlong_as_double(0x7ff8000000000000ll);
        if (HC && blockIdx.y == 0) {
            if (p.hash) p.hash[q] = 0;
            if (p.count) p.count[q] = 0;
        }
        return;
    }
    const uint64_t *Xq = p.X + q * (int64_t)p.d;
    Acc<PREC> acc[MC];
    uint64_t h = 0;
    int32_t cnt = 0;
    const bool paper = p.form == DDSG_FORM_PAPER;
    const int C = p.t.C;
    for (int c = 0; c < C; ++c) {
        const DevComp &cd = p.t.comps[c];
        const double b = cd.b;
        if (paper && b == 0.0) continue;
        const int k = cd.k;
        uint64_t Xd[KMAX];
        for (int j = 0; j < k; ++j) Xd[j] = Xq[cd.dims[j]];
        const int tb = paper ? cd.tup_begin : cd.tup_int;
        const int te = cd.tup_end;
        for (int ti = tb; ti < te; ++ti) {
            const DevTup tu = p.t.tups[ti];
            bool act = true;
            uint32_t off = 0;
            W w = (W)1;
            uint32_t cells[KMAX];
            for (int j = 0; j < k; ++j) {
                Basis1D o;
                const int l = tu.lev[j];
                if (!basis1d(Xd[j], l, o)) { act = false; break; }
                off = off * ncells(l) + o.cell;
                cells[j] = o.cell;
                if (PREC == DDSG_F64) w = w * ((W)__ull2double_rn(o.N) * pow2m_d(o.e));
                else w = w * ((W)__ull2float_rn(o.N) * pow2m_f(o.e));
            }
            if (!act) continue;
            const int32_t pid = p.t.slots[tu.slot_base + off];
            if (pid < 0) continue;
            if (paper) w = (W)b * w;
            if (PREC == DDSG_F64) {
                const double *a = p.t.alpha64 + (int64_t)pid * m + m0;
#pragma unroll
                for (int o = 0; o < MC; ++o)
                    if (m0 + o < m) acc[o].add(w, __ldg(a + o));
            } else {
                const float *a = p.t.alpha32 + (int64_t)pid * m + m0;
#pragma unroll
                for (int o = 0; o < MC; ++o)
                    if (m0 + o < m) acc[o].add(w, __ldg(a + o));
            }
            if (HC) {
                uint64_t z = (uint64_t)(uint32_t)c;
                for (int j = 0; j < k; ++j)
                    z = mix64(z ^ ((uint64_t)tu.lev[j] << 40) ^ (uint64_t)index_of_cell(tu.lev[j], cells[j]));
                h ^= mix64(z + 0x9E3779B97F4A7C15ull);
                ++cnt;
            }
        }
    }
#pragma unroll
    for (int o = 0; o < MC; ++o)
        if (m0 + o < m) p.y[q * m + m0 + o] = acc[o].result();
    if (HC && blockIdx.y == 0) {
        if (p.hash) p.hash[q] = h;
        if (p.count) p.count[q] = cnt;
    }
}

template <int PREC, int MC>
static cudaError_t launch_eval_mc(const EvalParams &p, bool hc, cudaStream_t st) {
    dim3 grid((unsigned)((p.n + 127) / 128), (unsigned)((p.m + MC - 1) / MC));
    if (hc) eval_lq_kernel<PREC, MC, true><<<grid, 128, 0, st>>>(p);
    else eval_lq_kernel<PREC, MC, false><<<grid, 128, 0, st>>>(p);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_eval_prec(const EvalParams &p, bool hc, cudaStream_t st) {
    if (p.m <= 1) return launch_eval_mc<PREC, 1>(p, hc, st);
    if (p.m <= 2) return launch_eval_mc<PREC, 2>(p, hc, st);
    if (p.m <= 4) return launch_eval_mc<PREC, 4>(p, hc, st);
    if (p.m <= 8) return launch_eval_mc<PREC, 8>(p, hc, st);
    if (p.m <= 12) return launch_eval_mc<PREC, 12>(p, hc, st);
    return launch_eval_mc<PREC, 16>(p, hc, st);
}

cudaError_t launch_eval(const EvalArgs &a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    EvalParams p;
    p.t = *a.t;
    p.d = a.d;
    p.m = a.m;
    p.n = a.n;
    p.X = a.X;
    p.flags = reinterpret_cast<const int32_t *>(a.X + a.n * (int64_t)a.d);
    p.y = a.y;
    p.hash = a.hash;
    p.count = a.count;
    p.form = a.form;
    const bool hc = a.hash != nullptr || a.count != nullptr;
    if (a.precision == DDSG_F64) return launch_eval_prec<DDSG_F64>(p, hc, st);
    return launch_eval_prec<DDSG_F32C>(p, hc, st);
}

// ---------------------------------------------------------------------------
// hierarchization: one block per component, layer by layer in level sum
// ---------------------------------------------------------------------------

constexpr int HC_CHUNK = 16;

__global__ void __launch_bounds__(128) hierarchize_kernel(const DevTables t, int m,
                                                          const double *__restrict__ values) {
    const DevComp cd = t.comps[blockIdx.x];
    const int k = cd.k;
    for (int s = 0; s < cd.nlayers; ++s) {
        const int lb = t.layer_off[cd.layer_begin + s];
        const int le = t.layer_off[cd.layer_begin + s + 1];
        const int npl = le - lb;
        const int nchunks = (m + HC_CHUNK - 1) / HC_CHUNK;
        for (int w = threadIdx.x; w < npl * nchunks; w += blockDim.x) {
            const int pl = w / nchunks;
            const int m0 = (w - pl * nchunks) * HC_CHUNK;
            const int pid = t.layer_pts[lb + pl];
            uint64_t Xp[KMAX];
            for (int j = 0; j < k; ++j)
                Xp[j] = node_X(t.pt_lv[(int64_t)j * t.P + pid], t.pt_ix[(int64_t)j * t.P + pid]);
            double acc[HC_CHUNK];
#pragma unroll
            for (int o = 0; o < HC_CHUNK; ++o) acc[o] = 0.0;
            for (int ti = cd.tup_begin; ti < cd.tup_end; ++ti) {
                const DevTup tu = t.tups[ti];
                if (tu.lsum >= s) continue;
                bool act = true;
                uint32_t off = 0;
                double wv = 1.0;
                for (int j = 0; j < k; ++j) {
                    Basis1D o;
                    if (!basis1d(Xp[j], tu.lev[j], o)) { act = false; break; }
                    off = off * ncells(tu.lev[j]) + o.cell;
                    wv *= __ull2double_rn(o.N) * pow2m_d(o.e);
                }
                if (!act) continue;
                const int32_t q = t.slots[tu.slot_base + off];
                if (q < 0) continue;
                const double *a = t.alpha64 + (int64_t)q * m + m0;
#pragma unroll
                for (int o = 0; o < HC_CHUNK; ++o)
                    if (m0 + o < m) acc[o] = fma(wv, a[o], acc[o]);
            }
#pragma unroll
            for (int o = 0; o < HC_CHUNK; ++o)
                if (m0 + o < m)
                    t.alpha64[(int64_t)pid * m + m0 + o] = values[(int64_t)pid * m + m0 + o] - acc[o];
        }
        __syncthreads();
    }
}

cudaError_t launch_hierarchize(const DevTables &t, int m, const double *values, cudaStream_t st) {
    if (t.C <= 0) return cudaSuccess;
    hierarchize_kernel<<<t.C, 128, 0, st>>>(t, m, values);
    return cudaGetLastError();
}

__global__ void to_f32_kernel(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __double2float_rn(a[i]);
}

cudaError_t launch_to_f32(const double *a, float *b, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    to_f32_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, b, n);
    return cudaGetLastError();
}

}  // namespace ddsg
