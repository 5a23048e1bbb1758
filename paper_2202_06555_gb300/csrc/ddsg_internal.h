// ddsg_internal.h -- private declarations shared by the libddsg translation units.
//
// Device data layout (all tables owned by the handle, uploaded by hdmr_hierarchize):
//
//   DevComp[C]        one per HDMR component u (eq. 4.2 index set):
//                       k, dims, b_u, tuple range [tup_begin, tup_end),
//                       first interior tuple (all levels >= 2) tup_int,
//                       point range [pt_begin, pt_end) and layer table offset.
//   DevTup[T]         one per non-empty level tuple of a component, ordered
//                       (interior flag, level sum, lexicographic): levels and the
//                       base offset of its dense cell directory in `slots`.
//   Device row order: per component, its tuples in DevTup order, and inside a
//   tuple its present cells in increasing cell index (last dim fastest).
//   pt_dpos[P]        device row of each point (points keep the caller's order).
//   mask (in DevTup)  presence bit per cell for tuples of <= 64 cells: the row of
//                       a cell is `first` + popcount of the present cells below it.
//   slots[S] int32    for larger tuples, a dense directory: for every cell the
//                       device row, or -1 if absent. Either way the support test
//                       of a query costs O(1) arithmetic per tuple (the
//                       per-level-tuple alternative to a tree walk).
//   alpha64[P*mp64]   FP64 surpluses by device row; rows padded with zeros to a
//                       multiple of 16 bytes so they load as double2.
//   alpha32[P*mp32]   FP32 copy used by the compensated FP32 form (float4 rows).
//   pt_lv/pt_ix       structure-of-arrays (level, index) tables, [KMAX][P].
//   layer_pts[P]      point ids of each component sorted by level sum, and
//   layer_off[...]    per component, the start of each level-sum layer in it
//                       (used by the layer-by-layer hierarchization).
//
// Query encoding (stored dimension-major, X[j*n + q], so that one coordinate
// of consecutive queries is contiguous): each canonical coordinate c in [0,1] is held as the 64-bit
// fixed-point integer X = floor(c * 2^62), with bit 0 forced to 1 when the
// product is not an integer (a sticky bit, so X never lands on a dyadic cell
// boundary unless c does). Cells, support tests and hash indices are then exact
// integer arithmetic; basis values are exact integers scaled by a power of two.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ddsg.h"

namespace ddsg {

constexpr int KMAX = DDSG_KMAX;
constexpr int LMAX = DDSG_LMAX;
constexpr uint64_t X_ONE = 1ull << 62;          // fixed-point 1.0
constexpr uint64_t X_NAN = 0xFFFFFFFFFFFFFFFFull; // marks a non-finite coordinate

struct DevComp {
    int32_t k;
    int32_t dims[KMAX];
    uint8_t lmax[KMAX];   // highest level present per dimension
    int32_t tup_begin, tup_int, tup_end;
    int32_t pt_begin, pt_end;
    int32_t layer_begin;  // index into layer_off; layers of this comp: layer_off[layer_begin .. +nlayers]
    int32_t nlayers;
    int32_t row_begin, row_int, row_end;  // device rows: all / interior (levels >= 2) / end
    double b;
};

struct DevTup {
    uint8_t lev[KMAX];
    int32_t first;      // device row of the tuple's first present point
    int32_t slot_base;  // cell directory offset, or -1 when the tuple has <= 64 cells
    int32_t lsum;       // sum of (l_j - 1)
    uint32_t nc1;       // cells of the second dimension's level (row stride of a 2D cell index)
    uint64_t mask;      // presence bit per cell when slot_base < 0
};

// Device row of cell `off` of tuple tu, or -1 if that cell holds no point.
// Rows of a tuple are stored in increasing cell order, so for tuples of <= 64
// cells the row is first + (number of present cells below off): no memory access.
__host__ __device__ inline int32_t tuple_row(const DevTup &tu, uint32_t off, const int32_t *slots) {
    if (tu.slot_base < 0) {
        if (!((tu.mask >> off) & 1ull)) return -1;
#ifdef __CUDA_ARCH__
        return tu.first + __popcll(tu.mask & ((2ull << off) - 1ull)) - 1;
#else
        return tu.first + __builtin_popcountll(tu.mask & ((2ull << off) - 1ull)) - 1;
#endif
    }
    return slots[tu.slot_base + off];
}

// ---------------------------------------------------------------------------
// Checked builds (-DDDSG_CHECKED): the bounds-checked stand-in for a memory
// sanitizer. Every table index a kernel derives from the tables is tested
// before the access it guards. A failed test sets its site's bit in the
// module's check word and the access is skipped: that query's result is wrong,
// but nothing is read or written out of bounds. Release builds compile every
// test to `true` (the expression is not even evaluated).
// ---------------------------------------------------------------------------
enum CheckSite : int {
    CK_CELL = 0,   // cell offset of a presence-mask tuple < 64
    CK_SLOT = 1,   // cell-directory index < S
    CK_ROW = 2,    // device row inside its component's rows
    CK_STAGE = 3,  // staged block inside its shared-memory buffer and the tables
    CK_DIM = 4,    // dimension index < d
    CK_POINT = 5,  // point id < P (hierarchization layers)
    CK_COMP = 6,   // component id < C (component lists)
    CK_NSITES = 7
};

#if defined(DDSG_CHECKED) && defined(__CUDACC__)
static __device__ unsigned long long g_check_word;   // one per module
__device__ __forceinline__ bool check_site(bool ok, int site) {
    if (!ok) atomicOr(&g_check_word, 1ull << site);
    return ok;
}
#define DDSG_CK(cond, site) ::ddsg::check_site((cond), (site))
#else
#define DDSG_CK(cond, site) true
#endif

#if defined(__CUDACC__)
// tuple_row with the checked-build tests: the cell offset of a presence-mask
// tuple, the directory index (S entries) and the row against [lo, hi), the
// rows of the tuple's component.
__device__ __forceinline__ int32_t tuple_row_at(const DevTup &tu, uint32_t off, const int32_t *slots,
                                                int64_t S, int32_t lo, int32_t hi) {
#if defined(DDSG_CHECKED)
    if (tu.slot_base < 0 ? !DDSG_CK(off < 64u, CK_CELL) : !DDSG_CK((int64_t)tu.slot_base + off < S, CK_SLOT))
        return -1;
    const int32_t r = tuple_row(tu, off, slots);
    return (r < 0 || DDSG_CK(r >= lo && r < hi, CK_ROW)) ? r : -1;
#else
    (void)S;
    (void)lo;
    (void)hi;
    return tuple_row(tu, off, slots);
#endif
}
#endif

// Check words of the modules with kernels, read and cleared (host; synchronous).
// Always 0 in release builds.
unsigned long long check_word_take_kernels();
unsigned long long check_word_take_irbc();

// Nodal-slab tables of one form for the staged nodal kernel (kernel 5, built on
// first use by ddsg_nodal.cu). A component's evaluated points (all of them in
// the paper form, the interior ones in the slice-free form) are grouped by
// their cell (b, cb) in the component's slab dimension; for every group the sum
// of its points' products is, as a function of the other (nodal) dimension, a
// piecewise-linear function with kinks on the grid of its finest level A, and
// is stored by its values at the 2^(A-1) + 1 nodes of that grid. A query then
// reads two adjacent node rows per slab level b instead of one row per level
// tuple. Components with k = 1 have one slab (no slab dimension); the constant
// component has one slab and A = 1.
//   meta       per component: nslab slab entries {b (0: no slab dimension),
//              offset of the slab's directory within the meta block}, then
//              the directory: per cell of each slab level {first node row
//              relative to the component's first row, or -1 if the cell holds
//              no point; A}. Each block is padded to a multiple of 16 bytes.
//   v64 / v32  node rows in FP64 (stride mp64) and FP32 (stride rs32).
struct DevNodal {
    int32_t ok = 0;            // built for the current tables (set by nodal_build)
    int32_t tried = 0;         // a build was attempted for the current tables
    int32_t vals = 0;          // node values computed from the current surpluses
    int32_t n = 0;             // processed components
    int64_t rows = 0;          // node rows
    int32_t rs32 = 0;          // FP32 row stride in floats (a multiple of 32 when m > 16)
    int32_t meta_bytes = 0;    // staged meta area (largest meta block, multiple of 128 bytes)
    int64_t stage_bytes[2] = {0, 0};  // staged bytes of the largest component per precision (meta + rows)
    int4 *rec = nullptr;       // per processed component: {meta begin (int2 units), nmeta | nslab << 16, first row, nrows}
    int4 *rec2 = nullptr;      // {component id, nodal dim | slab dim << 16 (0xffff: none), b_u, 0}
    int2 *meta = nullptr;
    double *v64 = nullptr;
    float *v32 = nullptr;
    // nodalization work: per node row {cell group, node index, A, 0}; per cell group
    // [begin, end) into gpts; per group point {surplus row, level, index, 0} in the nodal dimension
    int4 *nrow = nullptr;
    int2 *grp = nullptr;
    int4 *gpts = nullptr;
    int64_t ngrp = 0, ngpts = 0;
    double erows = 0;          // node rows a uniformly distributed query reads, summed over components
};

struct DevTables {
    int32_t C = 0, T = 0;
    int64_t P = 0, S = 0;
    int32_t m = 0;
    int32_t mp64 = 0;     // row stride of alpha64 (m rounded up to 2: 16-byte rows)
    int32_t mp32 = 0;     // row stride of alpha32 (m rounded up to 4: 16-byte rows)
    int32_t tile_ok = 0;  // every component fits the staged path (k <= 2, levels <= LT)
    DevComp *comps = nullptr;
    DevTup *tups = nullptr;
    int32_t *slots = nullptr;
    double *alpha64 = nullptr;
    float *alpha32 = nullptr;
    int32_t *layer_pts = nullptr;
    int32_t *layer_off = nullptr;
    uint8_t *pt_lv = nullptr;     // SoA levels:  pt_lv[j*P + p], j < KMAX
    uint32_t *pt_ix = nullptr;    // SoA indices: pt_ix[j*P + p]
    int32_t *pt_dpos = nullptr;   // device row of point p
    // components each form evaluates, in order (paper form skips b == 0), and
    // the largest surplus block (bytes, FP32 and FP64) one of them stages
    int32_t *proc[2] = {nullptr, nullptr};
    int32_t nproc[2] = {0, 0};
    // per processed component (same order), for the TMA-staged kernel:
    // {component, first staged row, rows | tuples << 20, first tuple}
    int4 *stage_rec[2] = {nullptr, nullptr};
    // dims[0] | dims[1] << 16 (dims[1] = dims[0] when k = 1; 0 when k = 0)
    uint32_t *pdims[2] = {nullptr, nullptr};
    int64_t stage_bytes[2][2] = {{0, 0}, {0, 0}};  // [form][precision]
    int32_t max_tuples = 0;                        // most level tuples in one component
    int32_t max_level = 0;                         // highest 1D level present anywhere
    DevNodal nod[2];                               // nodal-slab tables per form (kernel 5)
};

#if defined(__CUDACC__)
// Checked builds: component id c < C, with k <= KMAX and every dimension < d.
__device__ __forceinline__ bool comp_ok(const DevTables &t, int c, int d) {
#if defined(DDSG_CHECKED)
    if (!DDSG_CK(c >= 0 && c < t.C, CK_COMP)) return false;
    const DevComp &cd = t.comps[c];
    bool ok = cd.k >= 0 && cd.k <= KMAX;
    for (int j = 0; ok && j < cd.k; ++j) ok = cd.dims[j] >= 0 && cd.dims[j] < d;
    return DDSG_CK(ok, CK_DIM);
#else
    (void)t;
    (void)c;
    (void)d;
    return true;
#endif
}
#endif

// ---------------------------------------------------------------------------
// 1D basis on the fixed-point coordinate (boundary-augmented hats, Sec. 3.1)
// ---------------------------------------------------------------------------

__host__ __device__ inline uint32_t ncells(int l) {
    return l <= 1 ? 1u : (l == 2 ? 2u : (1u << (l - 2)));
}

// Cell of level l containing X, its support test (phi > 0 exactly) and the
// basis value numerator N with phi = N * 2^(-e). Returns active flag.
struct Basis1D {
    uint32_t cell;
    uint64_t N;
    int e;
};

__host__ __device__ inline bool basis1d(uint64_t X, int l, Basis1D &o) {
    if (l == 1) {
        o.cell = 0;
        o.N = 1;
        o.e = 0;
        return true;
    }
    if (l == 2) {
        // node 0 on [0, 1/2), node 1 on (1/2, 1]; phi = |2c - 1| = |X - 2^61| / 2^61
        const uint64_t half = 1ull << 61;
        o.cell = X >= half ? 1u : 0u;
        o.N = X >= half ? X - half : half - X;
        o.e = 61;
        return o.N != 0;
    }
    const int sh = 64 - l;                // cell width 2^sh in X units
    uint64_t cell = X >> sh;
    const uint64_t nmax = (1ull << (l - 2)) - 1;
    if (cell > nmax) cell = nmax;         // only at c = 1
    const uint64_t F = X - (cell << sh);  // position inside the cell, [0, 2^sh]
    const uint64_t half = 1ull << (sh - 1);
    const uint64_t dist = F >= half ? F - half : half - F;
    o.cell = (uint32_t)cell;
    o.N = half - dist;
    o.e = sh - 1;
    return o.N != 0;
}

__host__ __device__ inline uint32_t index_of_cell(int l, uint32_t cell) {
    return l == 1 ? 1u : (l == 2 ? 2u * cell : 2u * cell + 1u);
}

// fixed-point coordinate of node (l, i)
__host__ __device__ inline uint64_t node_X(int l, uint32_t i) {
    if (l == 1) return 1ull << 61;
    return (uint64_t)i << (63 - l);   // i / 2^(l-1) * 2^62
}

__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// kernel launchers (ddsg_kernels.cu)
// ---------------------------------------------------------------------------

// SM count of the current device (1 if it cannot be read): grid caps of the
// grid-stride kernels.
int device_sm_count();

cudaError_t launch_encode_queries(int64_t n, int d, const double *x, const double *lo,
                                  const double *span, uint64_t *X, int64_t *stats,
                                  cudaStream_t st);

constexpr int LT = 15;        // levels (1..LT) the staged evaluation path keeps per dimension

struct EvalConfig {
    int kernel = 0;           // 0 = tile kernel, 1 = per-tuple kernel, 2 = TMA-staged tile kernel
    int mc = 0;               // outputs per thread and pass (0 = heuristic)
};

constexpr int NKERNELS = 7;
constexpr int KERNEL_NODAL = 5;               // the staged nodal-slab kernel
constexpr int KERNEL_NODAL_TMEM = 6;          // the same, Kahan totals in tensor memory (FP32C)
inline bool kernel_is_nodal(int k) { return k == KERNEL_NODAL || k == KERNEL_NODAL_TMEM; }
constexpr int64_t TMA_STAGE_MAX = 84 * 1024;  // largest per-component surplus block staged by TMA
constexpr int TMA_TUP_MAX = 128;              // most level tuples of one component the staged kernel holds

struct EvalArgs {
    const DevTables *t;       // host copy of the table pointers
    int d, m;
    int64_t n;
    const uint64_t *X;        // d*n encoded queries (dimension-major), then n int32 flags
    double *y;                // n*m
    uint64_t *hash;           // nullable
    int32_t *count;           // nullable
    int form;                 // DDSG_FORM_*
    int precision;            // DDSG_F64 / DDSG_F32C
    EvalConfig cfg;
    unsigned long long *err = nullptr;  // device word: bounded waits that gave up (nullable)
    // failure-path test (hdmr_set_fault_injection): the staged kernels withhold the
    // staging copies of processed components >= withhold_from (-1: none)
    int withhold_from = -1;
};

// true if kernel `kernel` can run this handle/form/precision
bool eval_kernel_eligible(const DevTables &t, int kernel, int precision, int form);

// candidate output-chunk sizes the kernels are compiled for
int eval_mc_candidates(int precision, int kernel, int *out, int cap);

cudaError_t launch_eval(const EvalArgs &a, cudaStream_t st);

// Nodal-slab tables (ddsg_nodal.cu). Host view of one component for the planner.
struct NodalComp {
    int k;
    int32_t dims[KMAX];
    const uint8_t *lv;    // npts * k levels
    const uint32_t *ix;   // npts * k indices
    int64_t npts;
    int64_t first;        // global id of the component's first point
    double b;             // eq. 4.2 coefficient
};
// Plans and uploads the nodal tables of `form` into `out` (freed first). Tables
// the staged nodal kernel cannot hold leave out.ok = 0 and return DDSG_OK; a
// failed allocation or copy returns an error code (message set).
int nodal_build(int m, int form, const std::vector<NodalComp> &comps, const std::vector<int32_t> &dpos,
                DevNodal &out);
void nodal_free(DevNodal &nd);
// Node values from the FP64 surpluses, then their FP32 copy (asynchronous).
cudaError_t launch_nodalize(const DevNodal &nd, const double *alpha64, int mp64, int m, cudaStream_t st);
// true if the staged nodal kernel can run these tables (form, precision)
bool nodal_eligible(const DevTables &t, int precision, int form);
struct EvalParams;
cudaError_t launch_eval_nodal(const EvalParams &p, int precision, int mc, cudaStream_t st);
cudaError_t launch_eval_nodal_tmem(const EvalParams &p, cudaStream_t st);

cudaError_t launch_quadrature(const DevTables &t, int m, double *Q, cudaStream_t st);
cudaError_t launch_hierarchize(const DevTables &t, int m, const double *values,
                               cudaStream_t st);

// Read-only view of a hierarchized handle (host pointers to its device tables),
// for entry points defined outside ddsg_host.cu. Returns DDSG_OK or an error
// code with the message set (ddsg_last_error).
// The schedule in `cfg` is one the handle's current tables can run (an
// ineligible stored choice is reset to the default first, as hdmr_eval does).
struct HandleView {
    int d = 0, m = 0, device = -1;
    const DevTables *tables = nullptr;
    const double *lo = nullptr, *span = nullptr;
    int64_t *stats = nullptr;
    EvalConfig cfg;
    int withhold_from = -1;   // failure-path test switch of the handle
};
int handle_eval_view(hdmr_t *h, int precision, int form, HandleView *v);

// Event bracket (tracing on) around a launch made outside ddsg_host.cu, counted
// under `kind` in the handle's hdmr_profile_read totals like hdmr_eval's own.
struct HandleProfScope {
    hdmr_t *h;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    HandleProfScope(hdmr_t *h, int kind, cudaStream_t st);
    ~HandleProfScope();
};

// Event-based kernel tracer (host): brackets launches with CUDA events on the
// launching stream while enabled; read() waits for them and sums per kind.
struct Tracer {
    static constexpr int NK = 8;
    bool on = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[NK] = {0};
    int64_t n[NK] = {0};
    cudaEvent_t take() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
    }
    struct Scope {
        Tracer *t; int kind; cudaStream_t st; cudaEvent_t a = nullptr, b = nullptr;
        Scope(Tracer *t_, int k, cudaStream_t s) : t(t_), kind(k), st(s) {
            if (!t->on) return;
            a = t->take(); b = t->take();
            if (a) cudaEventRecord(a, st);
        }
        ~Scope() {
            if (!t->on || !a || !b) return;
            cudaEventRecord(b, st);
            t->recs.push_back({kind, a, b});
        }
    };
    void read(double *out_ms, int64_t *out_n, bool reset) {
        for (auto &r : recs) {
            float f = 0.f;
            if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&f, r.a, r.b) == cudaSuccess) {
                ms[r.kind] += f;
                n[r.kind] += 1;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
        for (int k = 0; k < NK; ++k) {
            if (out_ms) out_ms[k] = ms[k];
            if (out_n) out_n[k] = n[k];
            if (reset) { ms[k] = 0; n[k] = 0; }
        }
    }
    ~Tracer() {
        for (auto &r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};
int set_error(int code, const char *msg);

cudaError_t launch_to_f32(const double *a, int mp64, float *b, int mp32, int64_t P, int m,
                          cudaStream_t st);

}  // namespace ddsg
