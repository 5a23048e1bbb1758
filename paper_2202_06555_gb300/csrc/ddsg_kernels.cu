// ddsg_kernels.cu -- CUDA kernels of libddsg (sm_103a).
//
//   encode_queries   physical FP64 queries -> clamped canonical fixed point,
//                    transposed to dimension-major order through shared memory.
//   eval_tile        DDSG interpolation (Sec. 4.1, eq. 4.2 and the slice-free
//                    form): one thread per query, 128 queries per block, the
//                    block sweeps the components in lockstep so each
//                    component's tables stay hot in L1; per component the 1D
//                    basis of each of its dimensions is staged once per level in
//                    per-thread shared memory, then every non-empty level tuple
//                    costs one directory lookup; surplus rows load as 16-byte
//                    vectors into a chunk of MC output accumulators.
//   eval_lq          the same with the 1D basis recomputed per tuple (any k).
//   hierarchize      surpluses layer by layer (Sec. 3.1), one block per component.
#include <cuda_runtime.h>
#include <climits>
#include <stdint.h>

#include <type_traits>

#include "ddsg_internal.h"
#include "ddsg_eval.cuh"
#include "ddsg_tma.cuh"

namespace ddsg {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t point_key(int c, int k, const uint8_t *lev, const uint32_t *cells) {
    uint64_t z = (uint64_t)(uint32_t)c;
    for (int j = 0; j < k; ++j)
        z = mix64(z ^ ((uint64_t)lev[j] << 40) ^ (uint64_t)index_of_cell(lev[j], cells[j]));
    return mix64(z + 0x9E3779B97F4A7C15ull);
}

// ---------------------------------------------------------------------------
// query encoding (transposing)
// ---------------------------------------------------------------------------

// Block of 32x8 threads handles 32 queries; it loops over the d coordinates in
// tiles of 32, reading rows (coalesced along j) and writing X[j*n + q]
// (coalesced along q). flags[q] = 1 if any coordinate is non-finite.
__global__ void __launch_bounds__(256) encode_queries_kernel(int64_t n, int d, const double *__restrict__ x,
                                                             const double *__restrict__ lo,
                                                             const double *__restrict__ span,
                                                             uint64_t *__restrict__ X,
                                                             int32_t *__restrict__ flags,
                                                             unsigned long long *__restrict__ stats) {
    __shared__ uint64_t tile[32][33];
    __shared__ int bad_q[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
    unsigned long long clamps = 0;
    for (int64_t q0 = (int64_t)blockIdx.x * 32; q0 < n; q0 += (int64_t)gridDim.x * 32) {
        if (threadIdx.x < 32) bad_q[threadIdx.x] = 0;
        __syncthreads();
        for (int j0 = 0; j0 < d; j0 += 32) {
            // load: row r = query q0 + r, column tx = coordinate j0 + tx
            for (int r = ty; r < 32; r += 8) {
                const int64_t q = q0 + r;
                const int j = j0 + tx;
                uint64_t Xv = 0;
                if (q < n && j < d) {
                    const double xv = x[q * d + j];
                    double c = (xv - lo[j]) / span[j];
                    if (!isfinite(xv) || !isfinite(c)) {
                        Xv = X_NAN;
                        bad_q[r] = 1;
                    } else {
                        if (c < 0.0) { c = 0.0; ++clamps; }
                        if (c > 1.0) { c = 1.0; ++clamps; }
                        const double yv = c * 4611686018427387904.0;  // c * 2^62, exact
                        Xv = (uint64_t)yv;                              // floor (yv >= 0)
                        if ((double)Xv != yv) Xv |= 1ull;               // sticky bit
                    }
                }
                tile[r][tx] = Xv;
            }
            __syncthreads();
            // store: row = coordinate j0 + r, column tx = query q0 + tx
            for (int r = ty; r < 32; r += 8) {
                const int j = j0 + r;
                const int64_t q = q0 + tx;
                if (j < d && q < n) X[(int64_t)j * n + q] = tile[tx][r];
            }
            __syncthreads();
        }
        if (threadIdx.x < 32 && q0 + threadIdx.x < n) {
            flags[q0 + threadIdx.x] = bad_q[threadIdx.x];
            if (bad_q[threadIdx.x]) atomicAdd(&stats[1], 1ull);
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) clamps += __shfl_down_sync(0xffffffffu, clamps, o);
    if ((threadIdx.x & 31) == 0 && clamps) atomicAdd(&stats[0], clamps);
}

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

cudaError_t launch_encode_queries(int64_t n, int d, const double *x, const double *lo,
                                  const double *span, uint64_t *X, int64_t *stats,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int32_t *flags = reinterpret_cast<int32_t *>(X + n * (int64_t)d);
    int64_t blocks = (n + 31) / 32;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    encode_queries_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, d, x, lo, span, X, flags,
                                                           reinterpret_cast<unsigned long long *>(stats));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// evaluation
// ---------------------------------------------------------------------------

// acc[o] += w * alpha_row[m0 + o] for o < MC, reading 16-byte vectors; vectors
// past the padded row (stride mp) are skipped (never read).
template <int PREC, int MC>
__device__ __forceinline__ void accumulate(typename Types<PREC>::W (&acc)[MC], typename Types<PREC>::W w,
                                           const typename Types<PREC>::W *row, int m0, int mp) {
    using T = Types<PREC>;
    constexpr int VW = T::VW;
    const typename T::V *v = reinterpret_cast<const typename T::V *>(row + m0);
#pragma unroll
    for (int g = 0; g < MC / VW; ++g) {
        if (m0 + g * VW < mp) {
            const typename T::V a = __ldg(v + g);
            if constexpr (VW == 4) {
                acc[4 * g + 0] = fmaf(w, a.x, acc[4 * g + 0]);
                acc[4 * g + 1] = fmaf(w, a.y, acc[4 * g + 1]);
                acc[4 * g + 2] = fmaf(w, a.z, acc[4 * g + 2]);
                acc[4 * g + 3] = fmaf(w, a.w, acc[4 * g + 3]);
            } else {
                acc[2 * g + 0] = fma(w, a.x, acc[2 * g + 0]);
                acc[2 * g + 1] = fma(w, a.y, acc[2 * g + 1]);
            }
        }
    }
}

// Per-tuple evaluation of one component (any k), basis recomputed per tuple.
template <int PREC, int MC, bool HC>
__device__ __forceinline__ void comp_generic(const EvalParams &p, const DevComp &cd, int c,
                                             int64_t q, bool paper, int m0,
                                             typename Types<PREC>::W (&acc)[MC], uint64_t &h,
                                             int32_t &cnt) {
    using W = typename Types<PREC>::W;
    const int k = cd.k;
    uint64_t Xd[KMAX];
    for (int j = 0; j < k; ++j) Xd[j] = DDSG_CK(cd.dims[j] < p.d, CK_DIM) ? p.X[(int64_t)cd.dims[j] * p.n + q] : 0ull;
    const int tb = paper ? cd.tup_begin : cd.tup_int;
    const W *alpha = Types<PREC>::alpha(p.t);
    const int mp = Types<PREC>::stride(p.t);
    for (int ti = tb; ti < cd.tup_end; ++ti) {
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
            w = w * basis_val<W>(o);
        }
        if (!act) continue;
        const int32_t pid = tuple_row_at(tu, off, p.t.slots, p.t.S, cd.row_begin, cd.row_end);
        if (pid < 0) continue;
        if (paper) w = (W)cd.b * w;
        accumulate<PREC, MC>(acc, w, alpha + (int64_t)pid * mp, m0, mp);
        if (HC) {
            h ^= point_key(c, k, tu.lev, cells);
            ++cnt;
        }
    }
}

template <int PREC, int MC, bool HC>
__global__ void __launch_bounds__(128) eval_lq_kernel(const EvalParams p) {
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
    Result<PREC, MC> r;
    r.init();
    uint64_t h = 0;
    int32_t cnt = 0;
    const bool paper = p.form == DDSG_FORM_PAPER;
    for (int c = 0; c < p.t.C; ++c) {
        if (!comp_ok(p.t, c, p.d)) continue;
        const DevComp &cd = p.t.comps[c];
        if (paper && cd.b == 0.0) continue;
        comp_generic<PREC, MC, HC>(p, cd, c, q, paper, m0, r.partial(), h, cnt);
        r.fold();
    }
#pragma unroll
    for (int o = 0; o < MC; ++o)
        if (m0 + o < m) p.y[q * m + m0 + o] = r.value(o);
    if (HC && blockIdx.y == 0) {
        if (p.hash) p.hash[q] = h;
        if (p.count) p.count[q] = cnt;
    }
}

constexpr int TQ = 128;  // queries per block of the tile kernel

// Look up one level tuple for this thread's query from the staged 1D basis:
// device row (-1 if the query's cell holds no point or the query sits on a
// cell face) and the basis weight (0 when there is no point).
template <int PREC, int K>
__device__ __forceinline__ int32_t tile_probe(const DevTup &tu, const int32_t *slots, int64_t S, int32_t lo,
                                             int32_t hi, int tid,
                                             const uint32_t (*s_cell)[LT][TQ],
                                             const typename Types<PREC>::W (*s_t)[LT][TQ],
                                             typename Types<PREC>::W wb,
                                             typename Types<PREC>::W &w, uint32_t *cells) {
    using W = typename Types<PREC>::W;
    uint32_t off = 0;
    W wt = wb;
    if (K >= 1) {
        const uint32_t ca = s_cell[0][tu.lev[0] - 1][tid];
        cells[0] = ca;
        if (K == 1) {
            if (ca & 0x80000000u) { w = (W)0; return -1; }
            off = ca;
            wt = wb * s_t[0][tu.lev[0] - 1][tid];
        } else {
            const uint32_t cb = s_cell[1][tu.lev[1] - 1][tid];
            cells[1] = cb;
            if ((ca | cb) & 0x80000000u) { w = (W)0; return -1; }
            off = ca * tu.nc1 + cb;
            wt = wb * (s_t[0][tu.lev[0] - 1][tid] * s_t[1][tu.lev[1] - 1][tid]);
        }
    }
    const int32_t row = tuple_row_at(tu, off, slots, S, lo, hi);
    w = row >= 0 ? wt : (W)0;
    return row;
}

// Load the output chunk [m0, m0+MC) of device row `row` as 16-byte vectors
// (zeros when row < 0 or past the padded row).
template <int PREC, int MC>
__device__ __forceinline__ void tile_load(typename Types<PREC>::V (&v)[MC / Types<PREC>::VW],
                                          const typename Types<PREC>::W *alpha, int32_t row, int m0,
                                          int mp) {
    using T = Types<PREC>;
    const typename T::V *src = reinterpret_cast<const typename T::V *>(alpha + (int64_t)(row < 0 ? 0 : row) * mp + m0);
#pragma unroll
    for (int g = 0; g < MC / T::VW; ++g) {
        if (row >= 0 && m0 + g * T::VW < mp) v[g] = __ldg(src + g);
        else memset(&v[g], 0, sizeof(v[g]));
    }
}

template <int PREC, int MC>
__device__ __forceinline__ void tile_fma(typename Types<PREC>::W (&acc)[MC], typename Types<PREC>::W w,
                                         const typename Types<PREC>::V (&v)[MC / Types<PREC>::VW]) {
#pragma unroll
    for (int g = 0; g < MC / Types<PREC>::VW; ++g) {
        if constexpr (Types<PREC>::VW == 4) {
            acc[4 * g + 0] = fmaf(w, v[g].x, acc[4 * g + 0]);
            acc[4 * g + 1] = fmaf(w, v[g].y, acc[4 * g + 1]);
            acc[4 * g + 2] = fmaf(w, v[g].z, acc[4 * g + 2]);
            acc[4 * g + 3] = fmaf(w, v[g].w, acc[4 * g + 3]);
        } else {
            acc[2 * g + 0] = fma(w, v[g].x, acc[2 * g + 0]);
            acc[2 * g + 1] = fma(w, v[g].y, acc[2 * g + 1]);
        }
    }
}

// The tuples [tb, te) of one component with K dims, two at a time so that two
// surplus rows are in flight before their FMAs.
template <int PREC, int MC, bool HC, int K>
__device__ __forceinline__ void tile_tuples(const EvalParams &p, int c, int tb, int te,
                                            typename Types<PREC>::W wb, int m0, int tid,
                                            const uint32_t (*s_cell)[LT][TQ],
                                            const typename Types<PREC>::W (*s_t)[LT][TQ],
                                            typename Types<PREC>::W (&acc)[MC], uint64_t &h,
                                            int32_t &cnt) {
    using T = Types<PREC>;
    using W = typename T::W;
    const W *alpha = T::alpha(p.t);
    const int mp = T::stride(p.t);
#if defined(DDSG_CHECKED)
    const int32_t lo = p.t.comps[c].row_begin, hi = p.t.comps[c].row_end;
#else
    const int32_t lo = 0, hi = 0;
#endif
    for (int ti = tb; ti < te; ti += 2) {
        const bool two = ti + 1 < te;
        const DevTup t0 = p.t.tups[ti];
        const DevTup t1 = p.t.tups[two ? ti + 1 : ti];
        W w0, w1;
        uint32_t c0[2] = {0, 0}, c1[2] = {0, 0};
        const int32_t r0 = tile_probe<PREC, K>(t0, p.t.slots, p.t.S, lo, hi, tid, s_cell, s_t, wb, w0, c0);
        int32_t r1 = tile_probe<PREC, K>(t1, p.t.slots, p.t.S, lo, hi, tid, s_cell, s_t, wb, w1, c1);
        if (!two) {
            r1 = -1;
            w1 = (W)0;
        }
        typename T::V v0[MC / T::VW], v1[MC / T::VW];
        tile_load<PREC, MC>(v0, alpha, r0, m0, mp);
        tile_load<PREC, MC>(v1, alpha, r1, m0, mp);
        if constexpr (PREC == DDSG_F64) {   // FP64 issue slots are scarce: no FMAs on misses
            if (r0 >= 0) tile_fma<PREC, MC>(acc, w0, v0);
            if (r1 >= 0) tile_fma<PREC, MC>(acc, w1, v1);
        } else {
            tile_fma<PREC, MC>(acc, w0, v0);
            tile_fma<PREC, MC>(acc, w1, v1);
        }
        if (HC) {
            if (r0 >= 0) { h ^= point_key(c, K, t0.lev, c0); ++cnt; }
            if (r1 >= 0) { h ^= point_key(c, K, t1.lev, c1); ++cnt; }
        }
    }
}

template <int PREC, int MC, bool HC>
__global__ void __launch_bounds__(TQ) eval_tile_kernel(const EvalParams p) {
    using W = typename Types<PREC>::W;
    // staged 1D basis of the current component: [dim][level][thread]; bit 31 of
    // the cell marks "phi == 0 at this level" (query on a cell face).
    __shared__ uint32_t s_cell[2][LT][TQ];
    __shared__ W s_t[2][LT][TQ];
    const int tid = threadIdx.x;
    const int64_t q = (int64_t)blockIdx.x * TQ + tid;
    const int m0 = blockIdx.y * MC;
    const int m = p.m;
    const bool valid = q < p.n;
    const bool bad = !valid || p.flags[q] != 0;
    const bool paper = p.form == DDSG_FORM_PAPER;
    const W *alpha = Types<PREC>::alpha(p.t);
    const int mp = Types<PREC>::stride(p.t);
    Result<PREC, MC> r;
    r.init();
    uint64_t h = 0;
    int32_t cnt = 0;
    if (!bad) {
        for (int c = 0; c < p.t.C; ++c) {
            const DevComp &cd = p.t.comps[c];
            const double b = cd.b;
            if (paper && b == 0.0) continue;
            const int k = cd.k;
            if (k > 2 || cd.lmax[0] > LT || cd.lmax[1] > LT) {
                comp_generic<PREC, MC, HC>(p, cd, c, q, paper, m0, r.partial(), h, cnt);
                r.fold();
                continue;
            }
            // stage the 1D basis of each dimension, levels 1..lmax
            for (int j = 0; j < k; ++j) {
                const uint64_t Xv = DDSG_CK(cd.dims[j] < p.d, CK_DIM) ? p.X[(int64_t)cd.dims[j] * p.n + q] : 0ull;
                const int lm = cd.lmax[j];
                for (int l = 1; l <= lm; ++l) {
                    Basis1D o;
                    const bool act = basis1d(Xv, l, o);
                    s_cell[j][l - 1][tid] = act ? o.cell : 0x80000000u;
                    s_t[j][l - 1][tid] = basis_val<W>(o);
                }
            }
            const int tb = paper ? cd.tup_begin : cd.tup_int;
            const W wb = paper ? (W)b : (W)1;
            if (k == 2) tile_tuples<PREC, MC, HC, 2>(p, c, tb, cd.tup_end, wb, m0, tid, s_cell, s_t, r.partial(), h, cnt);
            else if (k == 1) tile_tuples<PREC, MC, HC, 1>(p, c, tb, cd.tup_end, wb, m0, tid, s_cell, s_t, r.partial(), h, cnt);
            else tile_tuples<PREC, MC, HC, 0>(p, c, tb, cd.tup_end, wb, m0, tid, s_cell, s_t, r.partial(), h, cnt);
            r.fold();
        }
    }
    if (!valid) return;
#pragma unroll
    for (int o = 0; o < MC; ++o)
        if (m0 + o < m) p.y[q * m + m0 + o] = bad ? __longlong_as_double(0x7ff8000000000000ll) : r.value(o);
    if (HC && blockIdx.y == 0) {
        if (p.hash) p.hash[q] = bad ? 0 : h;
        if (p.count) p.count[q] = bad ? 0 : cnt;
    }
}


// ---------------------------------------------------------------------------
// TMA-staged tile kernel (kernel 2: one warp group, 256 queries per block;
// kernel 3: two warp groups splitting each query's outputs, 192 queries per
// block). The surplus rows each component contributes (all rows, or the
// interior rows for the slice-free form) are one contiguous device-row range,
// copied into shared memory by a bulk TMA copy two components ahead.
// ---------------------------------------------------------------------------

// Block shape of the TMA-staged kernel with GR warp groups: QB queries per
// block; each query's output chunk is split over GR threads (one per group).
template <int GR>
struct TmaShape {
    static constexpr int QB = GR == 1 ? 256 : (GR == 2 ? 192 : 160);   // queries per block
    static constexpr int NT = QB * GR;               // threads per block
    static constexpr int QW = QB / 32;               // query warps per group
};

// shared memory before the staging buffers: barriers, per-query 1D basis
__host__ __device__ inline int tma_fixed_smem(int precision, int qb) {
    return 128 + (int)sizeof(uint16_t) * 2 * LT * qb + (precision == DDSG_F64 ? 8 : 4) * 2 * LT * qb;
}

// bytes of one staging buffer: component struct, its level tuples, its surplus rows
__host__ __device__ inline int tma_buf_bytes(int64_t stage) {
    return 128 + TMA_TUP_MAX * (int)sizeof(DevTup) + (int)((stage + 127) & ~127ll);
}

// shared memory of one probed tuple: a row index and a weight per query
inline int tma_probe_bytes(int precision, int qb) {
    return qb * (4 + (precision == DDSG_F64 ? 8 : 4));
}

// Staging buffers (3 when they fit, else 2) and probe batch (tuples probed per
// pass, at most the largest tuple count and TMA_PB_MAX) that fit in shared
// memory beside the fixed part; pb = 0 when not even two tuples fit.
inline void tma_layout(const DevTables &t, int fixed, int buf, int per, int &nbuf, int &pb, int min_pb = 2) {
    int want = t.max_tuples < 2 ? 2 : (t.max_tuples < TMA_PB_MAX ? t.max_tuples : TMA_PB_MAX);
    if (want < min_pb) want = min_pb;
    for (nbuf = TMA_NBUF_MAX; nbuf >= 2; --nbuf) {
        const int64_t left = (int64_t)kSmemLimit - fixed - (int64_t)nbuf * buf;
        pb = left > 0 ? (int)(left / per) : 0;
        if (pb > want) pb = want;
        if (pb >= (want < 8 ? want : 8) || nbuf == 2) break;
    }
    if (pb < min_pb) pb = 0;
}

// queries per block of evaluation kernel `kernel` (2, 3, 4: the TMA-staged kernel
// with 1, 2 or 3 warp groups)
static int tma_qb(int kernel) {
    return kernel == 4 ? TmaShape<3>::QB : (kernel == 3 ? TmaShape<2>::QB : TmaShape<1>::QB);
}

bool eval_kernel_eligible(const DevTables &t, int kernel, int precision, int form) {
    if (kernel == 0 || kernel == 1) return true;
    if (kernel == KERNEL_NODAL) return nodal_eligible(t, precision, form);
    if (kernel == KERNEL_NODAL_TMEM)
        return precision == DDSG_F32C && nodal_eligible(t, precision, form) && t.nod[form].rs32 % 32 == 0;
    if (kernel < 2 || kernel > 4) return false;
    if (!t.tile_ok) return false;   // the staged kernel handles only k <= 2, levels <= LT
    if (t.max_tuples > TMA_TUP_MAX) return false;
    const int qb = tma_qb(kernel);
    const int64_t bytes = t.stage_bytes[form][precision];
    if (bytes > TMA_STAGE_MAX) return false;
    int nbuf = 0, pb = 0;
    // the groups' point hashes are combined through the probe area: GR tuples at least
    tma_layout(t, tma_fixed_smem(precision, qb), tma_buf_bytes(bytes), tma_probe_bytes(precision, qb), nbuf, pb,
               kernel - 1 > 2 ? kernel - 1 : 2);
    return pb > 0;
}

// 1D basis of levels 1..lm at fixed-point coordinate X into staging slot j of
// query qi: cell (bit 15 = query on a face at that level) and hat value.
template <int PREC, int QB>
__device__ __forceinline__ void tma_stage(uint64_t X, int lm, int qi, uint16_t (*s_cell)[LT][QB],
                                          typename Types<PREC>::W (*s_t)[LT][QB], int j) {
    using W = typename Types<PREC>::W;
    s_cell[j][0][qi] = 0;
    s_t[j][0][qi] = (W)1;
    if (lm >= 2) {
        Basis1D o;
        const bool act = basis1d(X, 2, o);
        s_cell[j][1][qi] = act ? (uint16_t)o.cell : (uint16_t)0x8000u;
        s_t[j][1][qi] = basis_val<W>(o);
    }
    for (int l = 3; l <= lm; ++l) {
        // cell width 2^sh; position F in the cell; phi numerator N = min(F, 2^sh - F)
        const int sh = 64 - l;
        uint64_t cell = X >> sh;
        const uint64_t nmax = (1ull << (l - 2)) - 1;
        cell = cell > nmax ? nmax : cell;
        const uint64_t F = X - (cell << sh);
        const uint64_t R = (1ull << sh) - F;
        const uint64_t N = F < R ? F : R;
        s_cell[j][l - 1][qi] = N ? (uint16_t)cell : (uint16_t)0x8000u;
        if constexpr (PREC == DDSG_F64) s_t[j][l - 1][qi] = basis_to_f64(N, sh - 1);
        else s_t[j][l - 1][qi] = __uint2float_rn((uint32_t)(N >> (32 - l))) * pow2m_f(31);
    }
}

// Probe one level tuple for query qi: the staged row of the point whose
// support holds the query (-1 if there is none) and its weight
// wb * prod_j phi_j (zero on a miss). Selects instead of branches, apart from
// the warp-uniform test for a slot-directory tuple. A face flag (bit 15 of a
// staged cell) masks to cell 0, so off stays inside the tuple's cells.
template <int PREC, int K, int QB>
__device__ __forceinline__ int32_t tma_probe(const DevTup &tu, const int32_t *slots, int64_t S, int qi,
                                            const uint16_t (*s_cell)[LT][QB],
                                            const typename Types<PREC>::W (*s_t)[LT][QB],
                                            typename Types<PREC>::W wb, typename Types<PREC>::W &w,
                                            uint32_t *cells) {
    using W = typename Types<PREC>::W;
    uint32_t off = 0, face = 0;
    W wt = wb;
    if (K >= 1) {
        const uint32_t ca = s_cell[0][tu.lev[0] - 1][qi];
        cells[0] = ca;
        face = ca;
        off = ca & 0x7fffu;
        if (K == 1) {
            wt = wb * s_t[0][tu.lev[0] - 1][qi];
        } else {
            const uint32_t cb = s_cell[1][tu.lev[1] - 1][qi];
            cells[1] = cb;
            face |= cb;
            off = off * tu.nc1 + (cb & 0x7fffu);
            wt = wb * (s_t[0][tu.lev[0] - 1][qi] * s_t[1][tu.lev[1] - 1][qi]);
        }
    }
    int32_t row;
    if (tu.slot_base < 0) {
        const uint32_t o6 = off & 63u;
        const bool present = !(face & 0x8000u) && DDSG_CK(off < 64u, CK_CELL) && ((tu.mask >> o6) & 1ull);
        row = present ? tu.first + __popcll(tu.mask & ((2ull << o6) - 1ull)) - 1 : -1;
    } else {
        const int32_t s = DDSG_CK((int64_t)tu.slot_base + off < S, CK_SLOT) ? slots[tu.slot_base + off] : -1;
        row = (face & 0x8000u) ? -1 : s;
    }
    w = row >= 0 ? wt : (W)0;
    return row;
}

// Probe phase: tuples u = u0, u0 + du, ... below nb of stup for query qi. Per
// tuple the staged row to read goes to s_prow[u*QB + qi] and the weight to
// s_pw. The point hash and count of the parity checks are taken here. A miss
// has the weight zero and reads the tuple's first row (finite), so that the
// accumulate phase loads unconditionally.
template <int PREC, int K, bool HC, int QB>
__device__ __forceinline__ void tma_probe_batch(const EvalParams &p, int c, const DevTup *stup, int nb, int u0,
                                                int du, typename Types<PREC>::W wb, int qi,
                                                const uint16_t (*s_cell)[LT][QB],
                                                const typename Types<PREC>::W (*s_t)[LT][QB], int32_t row0,
                                                int32_t row_end, int32_t *s_prow, typename Types<PREC>::W *s_pw, uint64_t &h,
                                                int32_t &cnt) {
    using W = typename Types<PREC>::W;
#pragma unroll 4
    for (int u = u0; u < nb; u += du) {
        const DevTup &tu = stup[u];
        W w;
        uint32_t cl[2] = {0, 0};
        const int32_t row = tma_probe<PREC, K, QB>(tu, p.t.slots, p.t.S, qi, s_cell, s_t, wb, w, cl);
        const bool hit = row >= 0 && DDSG_CK(row >= row0 && row < row_end, CK_ROW);
        const int32_t first = DDSG_CK(tu.first >= row0 && tu.first < row_end, CK_ROW) ? tu.first : row0;
#if defined(DDSG_CHECKED)
        if (!hit) w = (W)0;
#else
        (void)row_end;
#endif
        s_prow[u * QB + qi] = (hit ? row : first) - row0;
        s_pw[u * QB + qi] = w;
        if (HC && hit) {
            h ^= point_key(c, K, tu.lev, cl);
            ++cnt;
        }
    }
}

// Accumulate phase: acc += w_u * row_u[m0, m0+MC) over the nb probed tuples,
// software-pipelined over two register slots. With U = 2 a slot holds one of
// the two rows of a step; with U = 1 (an output chunk too wide for two rows)
// slot 0 holds the first half of the row and slot 1 the second. Each slot is
// accumulated and at once refilled from the next step's row, so one slot's
// loads are in flight while the other's FMAs issue; the (row, weight) pairs
// are read two steps ahead. Row loads are unconditional (a miss reads a real,
// finite row with the weight zero); FULL: the chunk lies inside the padded row.
template <int PREC, int MC, bool FULL, int QB, int U>
__device__ __forceinline__ void tma_accumulate(const int32_t *s_prow, const typename Types<PREC>::W *s_pw,
                                               int nb, int qi, const typename Types<PREC>::W *sbuf, int m0,
                                               int mp, typename Types<PREC>::W (&acc)[MC]) {
    using T = Types<PREC>;
    using W = typename T::W;
    using V = typename T::V;
    constexpr int G = MC / T::VW;                                   // vectors per chunk
    constexpr int SV = U == 2 ? G : (G + 1) / 2;                    // vectors per slot
    V v[2][SV];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int g = 0; g < SV; ++g) memset(&v[s][g], 0, sizeof(v[s][g]));

    auto load_slot = [&](int s, int32_t rr) {
        const int g0 = U == 2 ? 0 : s * SV;
        const int ng = U == 2 ? G : (s == 0 ? SV : G - SV);
        const V *src = reinterpret_cast<const V *>(sbuf + (int64_t)rr * mp + m0);
#pragma unroll
        for (int g = 0; g < SV; ++g)
            if (g < ng && (FULL || m0 + (g0 + g) * T::VW < mp)) v[s][g] = src[g0 + g];
    };
    auto fma_slot = [&](int s, W wt) {
        const int g0 = U == 2 ? 0 : s * SV;
        const int ng = U == 2 ? G : (s == 0 ? SV : G - SV);
        if (PREC == DDSG_F64 && wt == (W)0) return;   // FP64 issues no FMA for a miss
#pragma unroll
        for (int g = 0; g < SV; ++g) {
            if (g < ng) {
                if constexpr (T::VW == 4) {
                    acc[4 * (g0 + g) + 0] = fmaf(wt, v[s][g].x, acc[4 * (g0 + g) + 0]);
                    acc[4 * (g0 + g) + 1] = fmaf(wt, v[s][g].y, acc[4 * (g0 + g) + 1]);
                    acc[4 * (g0 + g) + 2] = fmaf(wt, v[s][g].z, acc[4 * (g0 + g) + 2]);
                    acc[4 * (g0 + g) + 3] = fmaf(wt, v[s][g].w, acc[4 * (g0 + g) + 3]);
                } else {
                    acc[2 * (g0 + g) + 0] = fma(wt, v[s][g].x, acc[2 * (g0 + g) + 0]);
                    acc[2 * (g0 + g) + 1] = fma(wt, v[s][g].y, acc[2 * (g0 + g) + 1]);
                }
            }
        }
    };
    // (row, weight) of tuple t; past the batch: the last tuple's row, weight zero
    auto rd = [&](int t, int32_t &rr, W &ww) {
        const int tc = t < nb ? t : nb - 1;
        rr = s_prow[tc * QB + qi];
        const W x = s_pw[tc * QB + qi];
        ww = t < nb ? x : (W)0;
    };

    int32_t r1[U], r2[U];
    W w0[U], w1[U], w2[U];
#pragma unroll
    for (int u = 0; u < U; ++u) rd(u, r1[u], w0[u]);
#pragma unroll
    for (int s = 0; s < 2; ++s) load_slot(s, r1[U == 2 ? s : 0]);
#pragma unroll
    for (int u = 0; u < U; ++u) rd(U + u, r1[u], w1[u]);
    for (int t = 0; t < nb; t += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) rd(t + 2 * U + u, r2[u], w2[u]);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int u = U == 2 ? s : 0;
            fma_slot(s, w0[u]);
            load_slot(s, r1[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            w0[u] = w1[u];
            r1[u] = r2[u];
            w1[u] = w2[u];
        }
    }
}

// Barrier over the GR warps that share a query warp (named barrier 1 + qw);
// with the OR of `pred` over them. A single group needs none.
template <int GR>
__device__ __forceinline__ bool group_sync_or(int qw, bool pred) {
    if constexpr (GR == 1) {
        return pred;
    } else {
        uint32_t r;
        asm volatile(
            "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(r)
            : "r"((uint32_t)pred), "r"(1 + qw), "r"(32 * GR)
            : "memory");
        return r != 0;
    }
}
template <int GR>
__device__ __forceinline__ void group_sync(int qw) {
    if constexpr (GR > 1) asm volatile("barrier.sync %0, %1;" ::"r"(1 + qw), "r"(32 * GR) : "memory");
}

// Per evaluated component j, one TMA stage delivers into buffer j % nbuf:
//   [0, 96)                         the component struct,
//   [128, 128 + 32*TMA_TUP_MAX)     its level tuples (those the form evaluates),
//   [128 + 32*TMA_TUP_MAX, ...)     its surplus rows (one contiguous row range).
// full[b] completes when a stage has landed; empty[b] when every warp is done
// with it. Thread 0 stages component i+2 at the end of iteration i, into the
// buffer that component i+2-nbuf used: with nbuf = 3 warps may drift one
// component apart without a block barrier. Coordinates of component i+1 are
// loaded during component i from a per-component dims record, so no load
// stalls the start of a component.
// GR warp groups: group g handles outputs [m0 + g*MC, m0 + (g+1)*MC) of the
// same QB queries. With GR = 2 the two warps of a query warp split the work:
// group 0 stages dimension 0 and probes the even tuples, group 1 stages
// dimension 1 and probes the odd ones, both accumulate all tuples into their
// own outputs; a named barrier per warp pair orders staging, probing and
// accumulation. Every wait is bounded; a warp pair that gives up counts the
// timeout, marks its queries NaN and leaves the loop together (the OR over
// the pair is taken at its barrier), and before the block exits thread 0 waits
// (bounded) for the copies it issued.
template <int PREC, int MC, bool HC, int GR>
__global__ void __launch_bounds__(TmaShape<GR>::NT, 1) eval_tma_kernel(const EvalParams p, int buf_bytes, int nbuf,
                                                                        int pb) {
    using T = Types<PREC>;
    using W = typename T::W;
    constexpr int QB = TmaShape<GR>::QB;
    constexpr int QW = TmaShape<GR>::QW;
    constexpr int kWarps = TmaShape<GR>::NT / 32;
    // two rows in flight unless the output chunk alone fills the registers
    constexpr int U = (PREC == DDSG_F32C && MC * GR > 28) ? 1 : 2;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + TMA_NBUF_MAX;
    auto s_cell = reinterpret_cast<uint16_t (*)[LT][QB]>(smem + 128);
    auto s_t = reinterpret_cast<W (*)[LT][QB]>(smem + 128 + sizeof(uint16_t) * 2 * LT * QB);
    unsigned char *bufbase = smem + tma_fixed_smem(PREC, QB);
    int32_t *s_prow = reinterpret_cast<int32_t *>(bufbase + (size_t)nbuf * buf_bytes);
    W *s_pw = reinterpret_cast<W *>(s_prow + (size_t)pb * QB);
    constexpr int kTupOff = 128;
    constexpr int kRowOff = 128 + TMA_TUP_MAX * (int)sizeof(DevTup);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int grp = warp / QW;                 // output group of this thread
    const int qw = warp - grp * QW;            // query warp within the group
    const int qi = qw * 32 + lane;             // query within the block
    const int64_t q = (int64_t)blockIdx.x * QB + qi;
    const int64_t qc = q < p.n ? q : p.n - 1;   // clamped index for coordinate loads
    const int m0 = (blockIdx.y * GR + grp) * MC;
    const int m = p.m;
    const bool valid = q < p.n;
    const bool bad = !valid || p.flags[q] != 0;
    const bool paper = p.form == DDSG_FORM_PAPER;
    const int nproc = p.t.nproc[p.form];
    const int4 *recs = p.t.stage_rec[p.form];
    const uint32_t *pdims = p.t.pdims[p.form];
    const W *galpha = T::alpha(p.t);
    const int mp = T::stride(p.t);

    // thread 0: stage processed component j (record rec) into buffer j % nbuf
    // (a failure-path test withholds the copies from p.issue_end on)
    auto issue = [&](int j, int4 rec) {
        if (j >= p.issue_end) return;
        const int b = j % nbuf;
        const uint32_t nrows = (uint32_t)rec.z & 0xfffffu, nt = (uint32_t)rec.z >> 20;
        const uint32_t rbytes = nrows * (uint32_t)mp * (uint32_t)sizeof(W);
        const uint32_t tbytes = nt * (uint32_t)sizeof(DevTup);
        // (a failed test withholds the copy: the waits on it run out, the block writes NaN)
        if (!DDSG_CK(rec.x >= 0 && rec.x < p.t.C && nt <= (uint32_t)TMA_TUP_MAX &&
                         (int64_t)kRowOff + rbytes <= (int64_t)buf_bytes && rec.w >= 0 &&
                         (int64_t)rec.w + nt <= (int64_t)p.t.T && rec.y >= 0 && (int64_t)rec.y + nrows <= p.t.P,
                     CK_STAGE))
            return;
        unsigned char *dst = bufbase + (size_t)b * buf_bytes;
        mbar_expect_tx(&full[b], (uint32_t)sizeof(DevComp) + tbytes + rbytes);
        tma_bulk_g2s(dst, p.t.comps + rec.x, (uint32_t)sizeof(DevComp), &full[b]);
        if (tbytes) tma_bulk_g2s(dst + kTupOff, p.t.tups + rec.w, tbytes, &full[b]);
        if (rbytes) tma_bulk_g2s(dst + kRowOff, galpha + (int64_t)rec.y * mp, rbytes, &full[b]);
    };

    if (tid == 0) {
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], kWarps);
        }
        mbar_fence_init();
    }
    __syncthreads();
    int nissued = 0;
    int4 rec_next = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        if (nproc > 0) issue(0, recs[0]);
        if (nproc > 1) issue(1, recs[1]);
        nissued = nproc < 2 ? nproc : 2;
        if (nproc > 2) rec_next = recs[2];
    }

    Result<PREC, MC> r;
    r.init();
    uint64_t h = 0;
    int32_t cnt = 0;
    bool failed = false;
    int pfail = 0;                 // thread 0's refill wait gave up (warp-uniform)
    int staged0 = -1;              // dimension currently held in staging slot 0
    const int lmax_all = p.t.max_level < LT ? p.t.max_level : LT;
    uint64_t Xc0 = 0, Xc1 = 0;     // coordinates of the current component's dims
    uint32_t pd_next = 0;          // dims record of the next component
    if (nproc > 0) {
        const uint32_t pd = pdims[0];
        Xc0 = DDSG_CK((pd & 0xffffu) < (uint32_t)p.d, CK_DIM) ? p.X[(int64_t)(pd & 0xffffu) * p.n + qc] : 0ull;
        Xc1 = DDSG_CK((pd >> 16) < (uint32_t)p.d, CK_DIM) ? p.X[(int64_t)(pd >> 16) * p.n + qc] : 0ull;
    }
    if (nproc > 1) pd_next = pdims[1];
    int b = 0;
    uint32_t ph = 0;
    for (int i = 0; i < nproc; ++i) {
        uint64_t Xn0 = 0, Xn1 = 0;
        if (i + 1 < nproc) {
            Xn0 = DDSG_CK((pd_next & 0xffffu) < (uint32_t)p.d, CK_DIM) ? p.X[(int64_t)(pd_next & 0xffffu) * p.n + qc] : 0ull;
            Xn1 = DDSG_CK((pd_next >> 16) < (uint32_t)p.d, CK_DIM) ? p.X[(int64_t)(pd_next >> 16) * p.n + qc] : 0ull;
        }
        if (i + 2 < nproc) pd_next = pdims[i + 2];
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[b], ph));
        if (group_sync_or<GR>(qw, !ok || pfail)) {
            failed = true;
            if (lane == 0 && p.err) atomicAdd(p.err, 1ull);
            break;
        }
        const unsigned char *buf = bufbase + (size_t)b * buf_bytes;
        const DevComp &cd = *reinterpret_cast<const DevComp *>(buf);
        const int k = cd.k;
        if (!bad) {
            if (grp == 0 && k >= 1 && cd.dims[0] != staged0) {
                tma_stage<PREC, QB>(Xc0, k == 1 ? cd.lmax[0] : lmax_all, qi, s_cell, s_t, 0);
                staged0 = k == 1 ? -1 : cd.dims[0];
            }
            if (grp == GR - 1 && k == 2) tma_stage<PREC, QB>(Xc1, cd.lmax[1], qi, s_cell, s_t, 1);
        }
        const int c = HC ? p.t.proc[p.form][i] : 0;
        const int tb = paper ? cd.tup_begin : cd.tup_int;
        const int nt = cd.tup_end - tb;
        const int32_t row0 = paper ? cd.row_begin : cd.row_int;
        const W wb = paper ? (W)cd.b : (W)1;
        const DevTup *stup = reinterpret_cast<const DevTup *>(buf + kTupOff);
        const W *srow = reinterpret_cast<const W *>(buf + kRowOff);
        for (int t0 = 0; t0 < nt; t0 += pb) {
            const int nb = nt - t0 < pb ? nt - t0 : pb;
            group_sync<GR>(qw);   // staged basis visible; the partner is done with s_prow
            if (!bad) {
                if (k == 2) tma_probe_batch<PREC, 2, HC, QB>(p, c, stup + t0, nb, grp, GR, wb, qi, s_cell, s_t, row0, cd.row_end, s_prow, s_pw, h, cnt);
                else if (k == 1) tma_probe_batch<PREC, 1, HC, QB>(p, c, stup + t0, nb, grp, GR, wb, qi, s_cell, s_t, row0, cd.row_end, s_prow, s_pw, h, cnt);
                else tma_probe_batch<PREC, 0, HC, QB>(p, c, stup + t0, nb, grp, GR, wb, qi, s_cell, s_t, row0, cd.row_end, s_prow, s_pw, h, cnt);
            }
            group_sync<GR>(qw);   // the partner's probes visible
            if (!bad) {
                if (m0 + MC <= mp) tma_accumulate<PREC, MC, true, QB, U>(s_prow, s_pw, nb, qi, srow, m0, mp, r.partial());
                else tma_accumulate<PREC, MC, false, QB, U>(s_prow, s_pw, nb, qi, srow, m0, mp, r.partial());
            }
        }
        if (!bad) r.fold();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
        // producer: once every warp is done with component i+2-nbuf, stage i+2 in its buffer
        int pf = 0;
        if (tid == 0 && i + 2 < nproc) {
            const int j = i + 2;
            if (j >= nbuf && !mbar_wait_bounded(&empty[j % nbuf], (uint32_t)(((j - nbuf) / nbuf) & 1))) {
                pf = 1;
            } else {
                fence_proxy_async_smem();
                issue(j, rec_next);
                nissued = j + 1;
                if (j + 1 < nproc) rec_next = recs[j + 1];
            }
        }
        pfail = __shfl_sync(0xffffffffu, pf, 0);
        Xc0 = Xn0;
        Xc1 = Xn1;
        if (++b == nbuf) {
            b = 0;
            ph ^= 1u;
        }
    }
    __syncthreads();
    if (tid == 0) {
        // a block that gave up may still have copies in flight: let them land
        for (int j = nissued > nbuf ? nissued - nbuf : 0; j < nissued; ++j)
            if (j < p.issue_end) mbar_wait_bounded(&full[j % nbuf], (uint32_t)((j / nbuf) & 1));
    }
    if (HC && GR > 1) {
        // the point hash and count of a query are split over its groups: combine
        uint64_t *xh = reinterpret_cast<uint64_t *>(s_prow);
        int32_t *xc = reinterpret_cast<int32_t *>(xh + (GR - 1) * QB);
        if (grp > 0) {
            xh[(grp - 1) * QB + qi] = h;
            xc[(grp - 1) * QB + qi] = cnt;
        }
        __syncthreads();
        if (grp == 0) {
            for (int g = 0; g < GR - 1; ++g) {
                h ^= xh[g * QB + qi];
                cnt += xc[g * QB + qi];
            }
        }
    }
    if (!valid) return;
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int o = 0; o < MC; ++o)
        if (m0 + o < m) p.y[q * m + m0 + o] = (bad || failed) ? nanv : r.value(o);
    if (HC && blockIdx.y == 0 && grp == 0) {
        if (p.hash) p.hash[q] = (bad || failed) ? 0 : h;
        if (p.count) p.count[q] = (bad || failed) ? 0 : cnt;
    }
}

template <int PREC, int MC, int GR>
static cudaError_t launch_tma(const EvalParams &p, bool hc, cudaStream_t st) {
    constexpr int QB = TmaShape<GR>::QB, NT = TmaShape<GR>::NT;
    const int64_t stage = p.t.stage_bytes[p.form][PREC];
    const int buf = tma_buf_bytes(stage);
    int nbuf = 0, pb = 0;
    const int fixed = tma_fixed_smem(PREC, QB);
    tma_layout(p.t, fixed, buf, tma_probe_bytes(PREC, QB), nbuf, pb, GR > 2 ? GR : 2);
    const int smem = fixed + nbuf * buf + pb * tma_probe_bytes(PREC, QB);
    dim3 grid((unsigned)((p.n + QB - 1) / QB), (unsigned)((p.m + GR * MC - 1) / (GR * MC)));
    if (hc) {
        cudaError_t e = cudaFuncSetAttribute(eval_tma_kernel<PREC, MC, true, GR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        eval_tma_kernel<PREC, MC, true, GR><<<grid, NT, smem, st>>>(p, buf, nbuf, pb);
    } else {
        cudaError_t e = cudaFuncSetAttribute(eval_tma_kernel<PREC, MC, false, GR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        eval_tma_kernel<PREC, MC, false, GR><<<grid, NT, smem, st>>>(p, buf, nbuf, pb);
    }
    return cudaGetLastError();
}

// output chunks the two- and three-group kernels are compiled for (per group)
template <int PREC, int MC>
constexpr bool kGr2Chunk = PREC == DDSG_F64 ? (MC == 4 || MC == 8 || MC == 16) : (MC == 8 || MC == 16 || MC == 28);
template <int PREC, int MC>
constexpr bool kGr3Chunk = PREC == DDSG_F64 ? (MC == 4 || MC == 8) : (MC == 12 || MC == 20);

template <int PREC, int MC>
static cudaError_t launch_mc(const EvalParams &p, int kernel, bool hc, cudaStream_t st) {
    if constexpr (MC == 20) {   // compiled for the three-group kernel only
        if (kernel == 4) return launch_tma<PREC, MC, 3>(p, hc, st);
        return cudaErrorInvalidValue;
    } else {
    if (kernel == 2) return launch_tma<PREC, MC, 1>(p, hc, st);
    if (kernel == 3) {
        if constexpr (kGr2Chunk<PREC, MC>) return launch_tma<PREC, MC, 2>(p, hc, st);
        else return cudaErrorInvalidValue;
    }
    if (kernel == 4) {
        if constexpr (kGr3Chunk<PREC, MC>) return launch_tma<PREC, MC, 3>(p, hc, st);
        else return cudaErrorInvalidValue;
    }
    dim3 grid((unsigned)((p.n + TQ - 1) / TQ), (unsigned)((p.m + MC - 1) / MC));
    if (kernel == 0) {
        if (hc) eval_tile_kernel<PREC, MC, true><<<grid, TQ, 0, st>>>(p);
        else eval_tile_kernel<PREC, MC, false><<<grid, TQ, 0, st>>>(p);
    } else {
        if (hc) eval_lq_kernel<PREC, MC, true><<<grid, TQ, 0, st>>>(p);
        else eval_lq_kernel<PREC, MC, false><<<grid, TQ, 0, st>>>(p);
    }
    return cudaGetLastError();
    }
}

// compiled output-chunk sizes (multiples of the vector width)
static const int MC_F64[] = {2, 4, 6, 8, 12, 16};
static const int MC_F32[] = {4, 8, 12, 16, 28, 52};

// the two- and three-group TMA kernels (3, 4): chunks per group
static const int MC_F64_GR2[] = {4, 8, 16};
static const int MC_F32_GR2[] = {8, 16, 28};
static const int MC_F64_GR3[] = {4, 8};
static const int MC_F32_GR3[] = {12, 20};

// the nodal-slab kernel (5): 32 = the rotated two-window layout (FP32)
static const int MC_F64_NOD[] = {4, 8, 16};
static const int MC_F32_NOD[] = {32, 8, 16};

int eval_mc_candidates(int precision, int kernel, int *out, int cap) {
    const bool f64 = precision == DDSG_F64;
    if (kernel == KERNEL_NODAL) {
        const int *src = f64 ? MC_F64_NOD : MC_F32_NOD;
        for (int i = 0; i < 3 && i < cap; ++i) out[i] = src[i];
        return 3 < cap ? 3 : cap;
    }
    if (kernel == KERNEL_NODAL_TMEM) {   // FP32C only: 32-output windows
        if (cap < 1) return 0;
        out[0] = 32;
        return 1;
    }
    const int *src = kernel == 4 ? (f64 ? MC_F64_GR3 : MC_F32_GR3)
                     : kernel == 3 ? (f64 ? MC_F64_GR2 : MC_F32_GR2) : (f64 ? MC_F64 : MC_F32);
    const int n = kernel == 4 ? 2 : (kernel == 3 ? 3 : 6);
    for (int i = 0; i < n && i < cap; ++i) out[i] = src[i];
    return n < cap ? n : cap;
}

template <int PREC>
static cudaError_t launch_prec(const EvalParams &p, int kernel, int mc, bool hc, cudaStream_t st) {
    if constexpr (PREC == DDSG_F64) {
        switch (mc) {
            case 2: return launch_mc<PREC, 2>(p, kernel, hc, st);
            case 4: return launch_mc<PREC, 4>(p, kernel, hc, st);
            case 6: return launch_mc<PREC, 6>(p, kernel, hc, st);
            case 8: return launch_mc<PREC, 8>(p, kernel, hc, st);
            case 12: return launch_mc<PREC, 12>(p, kernel, hc, st);
            default: return launch_mc<PREC, 16>(p, kernel, hc, st);
        }
    } else {
        switch (mc) {
            case 4: return launch_mc<PREC, 4>(p, kernel, hc, st);
            case 8: return launch_mc<PREC, 8>(p, kernel, hc, st);
            case 12: return launch_mc<PREC, 12>(p, kernel, hc, st);
            case 16: return launch_mc<PREC, 16>(p, kernel, hc, st);
            case 20: return launch_mc<PREC, 20>(p, kernel, hc, st);
            case 28: return launch_mc<PREC, 28>(p, kernel, hc, st);
            default: return launch_mc<PREC, 52>(p, kernel, hc, st);
        }
    }
}

// Heuristic chunk: the smallest compiled size covering m, else the largest.
static int default_mc(int precision, int m) {
    int c[8];
    const int n = eval_mc_candidates(precision, 0, c, 8);
    for (int i = 0; i < n; ++i)
        if (c[i] >= m) return c[i];
    return precision == DDSG_F64 ? 16 : 28;
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
    p.err = a.err;
    p.issue_end = a.withhold_from < 0 ? INT_MAX : a.withhold_from;
    const bool hc = a.hash != nullptr || a.count != nullptr;
    EvalConfig cfg = a.cfg;
    if (kernel_is_nodal(cfg.kernel)) {
        // the nodal form has no per-point active set: hash / count requests
        // run the level-tuple tile kernel
        if (!hc) {
            if (cfg.kernel == KERNEL_NODAL_TMEM && a.precision == DDSG_F32C) return launch_eval_nodal_tmem(p, st);
            return launch_eval_nodal(p, a.precision, cfg.mc > 0 ? cfg.mc : (a.precision == DDSG_F64 ? 8 : 32), st);
        }
        cfg = EvalConfig();
    }
    const int mc = cfg.mc > 0 ? cfg.mc : default_mc(a.precision, a.m);
    if (a.precision == DDSG_F64) return launch_prec<DDSG_F64>(p, cfg.kernel, mc, hc, st);
    return launch_prec<DDSG_F32C>(p, cfg.kernel, mc, hc, st);
}

// ---------------------------------------------------------------------------
// hierarchization: one block per component, layer by layer in level sum
// ---------------------------------------------------------------------------

constexpr int HC_CHUNK = 16;

__global__ void __launch_bounds__(128) hierarchize_kernel(const DevTables t, int m,
                                                          const double *__restrict__ values) {
    const DevComp cd = t.comps[blockIdx.x];
    const int k = cd.k;
    const int mp = t.mp64;
    for (int s = 0; s < cd.nlayers; ++s) {
        const int lb = t.layer_off[cd.layer_begin + s];
        const int le = t.layer_off[cd.layer_begin + s + 1];
        const int npl = le - lb;
        const int nchunks = (m + HC_CHUNK - 1) / HC_CHUNK;
        for (int w = threadIdx.x; w < npl * nchunks; w += blockDim.x) {
            const int pl = w / nchunks;
            const int m0 = (w - pl * nchunks) * HC_CHUNK;
            const int pid = t.layer_pts[lb + pl];
            if (!DDSG_CK(pid >= 0 && pid < t.P && t.pt_dpos[pid] >= cd.row_begin && t.pt_dpos[pid] < cd.row_end,
                         CK_POINT))
                continue;
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
                    wv *= basis_to_f64(o.N, o.e);
                }
                if (!act) continue;
                const int32_t q = tuple_row_at(tu, off, t.slots, t.S, cd.row_begin, cd.row_end);
                if (q < 0) continue;
                const double *a = t.alpha64 + (int64_t)q * mp + m0;
#pragma unroll
                for (int o = 0; o < HC_CHUNK; ++o)
                    if (m0 + o < m) acc[o] = fma(wv, a[o], acc[o]);
            }
#pragma unroll
            for (int o = 0; o < HC_CHUNK; ++o)
                if (m0 + o < m)
                    t.alpha64[(int64_t)t.pt_dpos[pid] * mp + m0 + o] = values[(int64_t)pid * m + m0 + o] - acc[o];
        }
        __syncthreads();
    }
}

cudaError_t launch_hierarchize(const DevTables &t, int m, const double *values, cudaStream_t st) {
    if (t.C <= 0) return cudaSuccess;
    hierarchize_kernel<<<t.C, 128, 0, st>>>(t, m, values);
    return cudaGetLastError();
}

// Quadrature of every component interpolant (eq. 3.7): Q[c][o] = sum over the
// component's points (table order) of alpha_p[o] * prod_j int phi_{l_pj}, with
// int phi = 1 (level 1), 1/4 (level 2), 2^-(l-1) (level l >= 3). One thread per
// (component, output), FP64.
__global__ void quadrature_kernel(const DevTables t, int m, double *__restrict__ Q) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)t.C * m) return;
    const int c = (int)(e / m), o = (int)(e - (int64_t)c * m);
    const DevComp &cd = t.comps[c];
    double acc = 0.0;
    for (int64_t pnt = cd.pt_begin; pnt < cd.pt_end; ++pnt) {
        double w = 1.0;
        for (int j = 0; j < cd.k; ++j) {
            const int l = t.pt_lv[(int64_t)j * t.P + pnt];
            w *= l == 1 ? 1.0 : (l == 2 ? 0.25 : ldexp(1.0, -(l - 1)));
        }
        acc += w * t.alpha64[(int64_t)t.pt_dpos[pnt] * t.mp64 + o];
    }
    Q[e] = acc;
}

cudaError_t launch_quadrature(const DevTables &t, int m, double *Q, cudaStream_t st) {
    const int64_t n = (int64_t)t.C * m;
    quadrature_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(t, m, Q);
    return cudaGetLastError();
}

__global__ void to_f32_kernel(const double *__restrict__ a, int mp64, float *__restrict__ b, int mp32,
                              int64_t P, int m) {
    const int64_t total = P * (int64_t)mp32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pt = i / mp32;
        const int j = (int)(i - pt * mp32);
        b[i] = j < m ? __double2float_rn(a[pt * mp64 + j]) : 0.0f;
    }
}

cudaError_t launch_to_f32(const double *a, int mp64, float *b, int mp32, int64_t P, int m,
                          cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    int64_t blocks = (P * mp32 + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 32;
    if (blocks > cap) blocks = cap;
    to_f32_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, mp64, b, mp32, P, m);
    return cudaGetLastError();
}

// Check word of this module, read and cleared (all bits set if it cannot be read).
unsigned long long check_word_take_kernels() {
#if defined(DDSG_CHECKED)
    unsigned long long w = 0;
    const unsigned long long z = 0;
    if (cudaMemcpyFromSymbol(&w, g_check_word, sizeof w) != cudaSuccess ||
        cudaMemcpyToSymbol(g_check_word, &z, sizeof z) != cudaSuccess) {
        cudaGetLastError();
        return ~0ull;
    }
    return w;
#else
    return 0;
#endif
}

}  // namespace ddsg
