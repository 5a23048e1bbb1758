// ddsg_host.cu -- host runtime of libddsg: the hdmr_t handle, grid tables,
// validation, eq. 4.2 coefficients, refinement (eq. 3.8), upload and launches.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include <atomic>

#include "ddsg_alloc.h"
#include "ddsg_internal.h"
#include "ddsg_io.h"
#include "ddsg_tables.h"

using namespace ddsg;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(DDSG_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                              \
    } while (0)

extern "C" const char *ddsg_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// device allocation with the failure switch
// ---------------------------------------------------------------------------

static std::atomic<int> g_alloc_skip{0}, g_alloc_fail{0};

cudaError_t ddsg::dev_alloc(void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (g_alloc_fail.load() > 0) {
        if (g_alloc_skip.load() > 0) {
            g_alloc_skip.fetch_sub(1);
        } else {
            g_alloc_fail.fetch_sub(1);
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(ptr, bytes);
}

extern "C" int ddsg_inject_alloc_failure(int skip, int count) {
    if (skip < 0 || count < 0) return fail(DDSG_ERR_ARG, "ddsg_inject_alloc_failure: negative argument");
    g_alloc_skip.store(count ? skip : 0);
    g_alloc_fail.store(count);
    return DDSG_OK;
}

#define ALLOC_TRY(ptr, bytes, what)                                                       \
    do {                                                                                  \
        if (dev_alloc((ptr), (bytes)) != cudaSuccess) {                                   \
            cudaGetLastError();                                                           \
            return fail(DDSG_ERR_OOM, "%s: %zu bytes of device memory unavailable", (what), \
                        (size_t)(bytes));                                                 \
        }                                                                                 \
    } while (0)
#if defined(DDSG_CHECKED)
extern "C" const char *ddsg_version(void) { return "libddsg 0.1 (sm_103a, checked)"; }
extern "C" int ddsg_checked_build(void) { return 1; }
#else
extern "C" const char *ddsg_version(void) { return "libddsg 0.1 (sm_103a)"; }
extern "C" int ddsg_checked_build(void) { return 0; }
#endif

extern "C" int ddsg_take_check_word(uint64_t *word) {
    if (!word) return fail(DDSG_ERR_ARG, "ddsg_take_check_word: NULL argument");
    *word = check_word_take_kernels() | check_word_take_irbc();
    return DDSG_OK;
}

#if defined(DDSG_CHECKED)
static const char *const kCheckSiteName[CK_NSITES] = {"cell", "slot", "row", "stage", "dim", "point", "component"};
#endif

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------

struct Comp {
    int k = 0;
    int32_t dims[KMAX];
    std::vector<uint8_t> lv;   // npts * k
    std::vector<uint32_t> ix;  // npts * k
    int64_t npts() const { return k == 0 ? (int64_t)lv.size() : (int64_t)lv.size() / k; }
};

struct hdmr {
    int d = 0, m = 0, order = 0, device = 0;
    std::vector<double> anchor, lo, hi, span;
    bool anchor_central = false;
    bool closed = false;      // accepted set downward closed (set at upload)
    std::vector<Comp> comps;
    std::vector<int64_t> first_point;  // per comp, offset in concatenated order
    int64_t P = 0;
    // device state
    DevTables dt;
    bool uploaded = false;    // dt matches comps
    bool have_alpha = false;  // alpha64/alpha32 valid
    std::vector<double> b;
    std::vector<int32_t> dpos;  // device row of each point (host copy)
    std::vector<int32_t> ntup[2];   // level tuples per component walked in each form (set at upload)
    double *dlo = nullptr, *dspan = nullptr;
    int64_t *stats = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *hbuf = nullptr;      // device staging for hdmr_eval_host
    size_t hbuf_bytes = 0;
    // evaluation kernel choice per [precision][form] (autotuned or heuristic)
    EvalConfig cfg[2][2];
    // graph replay of hdmr_eval_graph: one cached executable graph for the
    // last (n, x, y, precision, form, schedule, table generation), replayed on
    // a handle-owned stream ordered against the caller's stream by events
    int fi_withhold = -1;           // failure-path test (hdmr_set_fault_injection)
    uint64_t gen = 1;               // bumped whenever a captured pointer may change
    bool capturing = false;         // ProfScope records nothing while capturing
    cudaGraphExec_t gexec = nullptr;
    int64_t g_n = -1;
    const double *g_x = nullptr;
    double *g_y = nullptr;
    int g_prec = -1, g_form = -1;
    EvalConfig g_cfg;
    uint64_t g_gen = 0;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    // tracing
    bool prof = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[DDSG_NKINDS] = {0};
    int64_t prof_n[DDSG_NKINDS] = {0};
};

// Event bracket around one launch when tracing is on.
struct ProfScope {
    hdmr *h;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    static cudaEvent_t take(hdmr *h) {
        if (!h->pool.empty()) {
            cudaEvent_t e = h->pool.back();
            h->pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    ProfScope(hdmr *h_, int kind_, cudaStream_t st_) : h(h_), kind(kind_), st(st_) {
        if (!h->prof || h->capturing) return;
        a = take(h);
        b = take(h);
        if (a) cudaEventRecord(a, st);
    }
    ~ProfScope() {
        if (!h->prof || !a || !b) return;
        cudaEventRecord(b, st);
        h->recs.push_back({kind, a, b});
    }
};

// Keeps the caller's current device, switches to the handle's for the call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static void free_tables(DevTables &t) {
    cudaFree(t.comps);
    cudaFree(t.tups);
    cudaFree(t.slots);
    cudaFree(t.alpha64);
    cudaFree(t.alpha32);
    cudaFree(t.layer_pts);
    cudaFree(t.layer_off);
    cudaFree(t.pt_lv);
    cudaFree(t.pt_ix);
    cudaFree(t.pt_dpos);
    cudaFree(t.proc[0]);
    cudaFree(t.proc[1]);
    cudaFree(t.stage_rec[0]);
    cudaFree(t.stage_rec[1]);
    cudaFree(t.pdims[0]);
    cudaFree(t.pdims[1]);
    nodal_free(t.nod[0]);
    nodal_free(t.nod[1]);
    t = DevTables();
}

// First GPU use: bind the handle to the current device and allocate its
// small per-handle buffers (domain map, counters).
static int ensure_device(hdmr *h) {
    if (h->device >= 0) return DDSG_OK;
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    const int d = h->d;
    // a failed allocation leaves the handle unbound, with nothing held
    auto undo = [h] {
        cudaFree(h->dlo);
        cudaFree(h->dspan);
        cudaFree(h->stats);
        h->dlo = h->dspan = nullptr;
        h->stats = nullptr;
    };
    if (dev_alloc(&h->dlo, sizeof(double) * d) != cudaSuccess ||
        dev_alloc(&h->dspan, sizeof(double) * d) != cudaSuccess ||
        dev_alloc(&h->stats, sizeof(int64_t) * 4) != cudaSuccess) {
        cudaGetLastError();
        undo();
        return fail(DDSG_ERR_OOM, "first device use: per-handle buffers unavailable");
    }
    CUDA_TRY(cudaMemcpy(h->dlo, h->lo.data(), sizeof(double) * d, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(h->dspan, h->span.data(), sizeof(double) * d, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(h->stats, 0, sizeof(int64_t) * 4));
    h->device = dev;
    return DDSG_OK;
}

extern "C" int hdmr_create(int d, int m, int order, const double *anchor, const double *lo,
                           const double *hi, hdmr_t **out) {
    if (!out) return fail(DDSG_ERR_ARG, "hdmr_create: out is NULL");
    *out = nullptr;
    if (d < 1 || m < 1 || order < 0 || order > KMAX)
        return fail(DDSG_ERR_ARG, "hdmr_create: need d >= 1, m >= 1, 0 <= order <= %d", KMAX);
    if (!anchor || !lo || !hi) return fail(DDSG_ERR_ARG, "hdmr_create: NULL anchor/lo/hi");
    hdmr *h = new (std::nothrow) hdmr();
    if (!h) return fail(DDSG_ERR_OOM, "hdmr_create: host allocation failed");
    h->d = d;
    h->m = m;
    h->order = order;
    h->anchor.assign(anchor, anchor + d);
    h->lo.assign(lo, lo + d);
    h->hi.assign(hi, hi + d);
    h->span.resize(d);
    h->anchor_central = true;
    for (int i = 0; i < d; ++i) {
        if (!(lo[i] < hi[i])) {
            delete h;
            return fail(DDSG_ERR_ARG, "hdmr_create: lo[%d] < hi[%d] required", i, i);
        }
        h->span[i] = hi[i] - lo[i];
        if ((anchor[i] - lo[i]) / h->span[i] != 0.5) h->anchor_central = false;
    }
    h->device = -1;  // bound to the current device at first GPU use
    *out = h;
    return DDSG_OK;
}

extern "C" int hdmr_destroy(hdmr_t *h) {
    if (!h) return DDSG_OK;
    if (h->device < 0) {
        delete h;
        return DDSG_OK;
    }
    DeviceGuard g(h->device);
    free_tables(h->dt);
    cudaFree(h->dlo);
    cudaFree(h->dspan);
    cudaFree(h->stats);
    cudaFree(h->ws);
    cudaFree(h->hbuf);
    for (auto &r : h->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : h->pool) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    for (auto e : h->gev)
        if (e) cudaEventDestroy(e);
    delete h;
    return DDSG_OK;
}

// ---------------------------------------------------------------------------
// components
// ---------------------------------------------------------------------------

static bool valid_index(int l, uint32_t i) {
    if (l == 1) return i == 1;
    if (l == 2) return i == 0 || i == 2;
    return (i & 1u) && i < (1u << (l - 1));
}

static uint32_t cell_of_index(int l, uint32_t i) {
    return l == 1 ? 0u : (l == 2 ? i / 2 : (i - 1) / 2);
}

static int level_sum(const uint8_t *lv, int k) {
    int s = 0;
    for (int j = 0; j < k; ++j) s += lv[j] - 1;
    return s;
}

static std::string point_key(const uint8_t *lv, const uint32_t *ix, int k) {
    std::string s;
    s.append(reinterpret_cast<const char *>(lv), k);
    s.append(reinterpret_cast<const char *>(ix), sizeof(uint32_t) * k);
    return s;
}

static void rebuild_offsets(hdmr *h) {
    h->first_point.resize(h->comps.size());
    int64_t off = 0;
    for (size_t c = 0; c < h->comps.size(); ++c) {
        h->first_point[c] = off;
        off += h->comps[c].npts();
    }
    h->P = off;
}

extern "C" int hdmr_add_component(hdmr_t *h, int k, const int32_t *dims, int64_t npts,
                                  const uint8_t *levels, const uint32_t *indices,
                                  int32_t *comp_id) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_add_component: NULL handle");
    if (k < 0 || k > h->order) return fail(DDSG_ERR_ARG, "hdmr_add_component: k=%d outside [0, order=%d]", k, h->order);
    if (npts < 1) return fail(DDSG_ERR_ARG, "hdmr_add_component: npts must be >= 1");
    if (k == 0 && npts != 1) return fail(DDSG_ERR_ARG, "hdmr_add_component: the empty component has exactly 1 point");
    if (k > 0 && (!dims || !levels || !indices)) return fail(DDSG_ERR_ARG, "hdmr_add_component: NULL table");
    if (npts > (int64_t)1 << 30) return fail(DDSG_ERR_ARG, "hdmr_add_component: too many points");
    Comp c;
    c.k = k;
    for (int j = 0; j < KMAX; ++j) c.dims[j] = -1;
    for (int j = 0; j < k; ++j) {
        if (dims[j] < 0 || dims[j] >= h->d) return fail(DDSG_ERR_ARG, "hdmr_add_component: dim %d out of range", dims[j]);
        if (j > 0 && dims[j] <= dims[j - 1]) return fail(DDSG_ERR_ARG, "hdmr_add_component: dims must be strictly ascending");
        c.dims[j] = dims[j];
    }
    for (const Comp &o : h->comps) {
        if (o.k == k && std::equal(o.dims, o.dims + k, c.dims))
            return fail(DDSG_ERR_ARG, "hdmr_add_component: component already present");
    }
    if (k == 0) {
        c.lv.assign(1, 0);  // one point, zero dims (size 1 marker)
        c.ix.assign(1, 0);
    } else {
        c.lv.assign(levels, levels + npts * k);
        c.ix.assign(indices, indices + npts * k);
        std::unordered_map<std::string, int64_t> seen;
        seen.reserve((size_t)npts * 2);
        for (int64_t p = 0; p < npts; ++p) {
            for (int j = 0; j < k; ++j) {
                int l = c.lv[p * k + j];
                if (l < 1 || l > LMAX) return fail(DDSG_ERR_TABLE, "hdmr_add_component: point %lld dim %d level %d outside [1,%d]", (long long)p, j, l, LMAX);
                if (!valid_index(l, c.ix[p * k + j])) return fail(DDSG_ERR_TABLE, "hdmr_add_component: point %lld dim %d index %u invalid for level %d", (long long)p, j, c.ix[p * k + j], l);
            }
            if (!seen.emplace(point_key(&c.lv[p * k], &c.ix[p * k], k), p).second)
                return fail(DDSG_ERR_TABLE, "hdmr_add_component: duplicate point %lld", (long long)p);
        }
    }
    h->comps.push_back(std::move(c));
    rebuild_offsets(h);
    h->uploaded = false;
    h->have_alpha = false;
    if (comp_id) *comp_id = (int32_t)h->comps.size() - 1;
    return DDSG_OK;
}

// Regular grid of eq. 3.5: all level tuples with sum(l-1) <= L-1, canonical order.
static void gen_compositions(int k, int s, std::vector<std::vector<int>> &out) {
    // compositions of s into k non-negative parts, lexicographic
    std::vector<int> e(k, 0);
    std::function<void(int, int)> rec;
    rec = [&](int j, int rest) {
        if (j == k - 1) {
            e[j] = rest;
            out.push_back(e);
            return;
        }
        for (int v = 0; v <= rest; ++v) {
            e[j] = v;
            rec(j + 1, rest - v);
        }
    };
    if (k == 0) {
        if (s == 0) out.push_back(e);
        return;
    }
    rec(0, s);
}

extern "C" int hdmr_add_regular_component(hdmr_t *h, int k, const int32_t *dims, int level,
                                          int32_t *comp_id) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_add_regular_component: NULL handle");
    if (level < 1 || level > LMAX) return fail(DDSG_ERR_ARG, "hdmr_add_regular_component: level out of range");
    if (k == 0) return hdmr_add_component(h, 0, dims, 1, nullptr, nullptr, comp_id);
    std::vector<uint8_t> lv;
    std::vector<uint32_t> ix;
    for (int s = 0; s <= level - 1; ++s) {
        std::vector<std::vector<int>> comps;
        gen_compositions(k, s, comps);
        for (auto &e : comps) {
            std::vector<uint32_t> n(k);
            uint64_t tot = 1;
            for (int j = 0; j < k; ++j) {
                n[j] = ncells(e[j] + 1);
                tot *= n[j];
            }
            if (tot > (1ull << 28) || lv.size() / k + tot > (1ull << 30))
                return fail(DDSG_ERR_ARG, "hdmr_add_regular_component: grid too large");
            std::vector<uint32_t> r(k, 0);
            for (uint64_t t = 0; t < tot; ++t) {
                for (int j = 0; j < k; ++j) {
                    lv.push_back((uint8_t)(e[j] + 1));
                    ix.push_back(index_of_cell(e[j] + 1, r[j]));
                }
                for (int j = k - 1; j >= 0; --j) {  // last dim fastest
                    if (++r[j] < n[j]) break;
                    r[j] = 0;
                }
            }
        }
    }
    return hdmr_add_component(h, k, dims, (int64_t)(lv.size() / k), lv.data(), ix.data(), comp_id);
}

extern "C" int hdmr_num_components(const hdmr_t *h, int32_t *ncomp, int64_t *npts) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_num_components: NULL handle");
    if (ncomp) *ncomp = (int32_t)h->comps.size();
    if (npts) *npts = h->P;
    return DDSG_OK;
}

extern "C" int hdmr_component_info(const hdmr_t *h, int32_t comp, int32_t *k, int32_t *dims,
                                   int64_t *npts, int64_t *first_point) {
    if (!h || comp < 0 || comp >= (int32_t)h->comps.size())
        return fail(DDSG_ERR_ARG, "hdmr_component_info: bad handle or component");
    const Comp &c = h->comps[comp];
    if (k) *k = c.k;
    if (dims) for (int j = 0; j < KMAX; ++j) dims[j] = c.dims[j];
    if (npts) *npts = c.npts();
    if (first_point) *first_point = h->first_point[comp];
    return DDSG_OK;
}

extern "C" int hdmr_component_points(const hdmr_t *h, int32_t comp, int64_t first, int64_t count,
                                     uint8_t *levels, uint32_t *indices, double *coords) {
    if (!h || comp < 0 || comp >= (int32_t)h->comps.size())
        return fail(DDSG_ERR_ARG, "hdmr_component_points: bad handle or component");
    const Comp &c = h->comps[comp];
    if (first < 0 || count < 0 || first + count > c.npts())
        return fail(DDSG_ERR_ARG, "hdmr_component_points: range outside the component");
    const int k = c.k;
    for (int64_t p = first; p < first + count; ++p) {
        for (int j = 0; j < k; ++j) {
            const int l = c.lv[p * k + j];
            const uint32_t i = c.ix[p * k + j];
            const int64_t o = (p - first) * k + j;
            if (levels) levels[o] = (uint8_t)l;
            if (indices) indices[o] = i;
            if (coords) {
                const double xc = (l == 1) ? 0.5 : ldexp((double)i, -(l - 1));
                const int dm = c.dims[j];
                coords[o] = h->lo[dm] + xc * h->span[dm];
            }
        }
    }
    return DDSG_OK;
}

// ---------------------------------------------------------------------------
// table upload: closure check, eq. 4.2 coefficients, tuple directories, layers
// ---------------------------------------------------------------------------

static std::vector<int32_t> dims_vec(const Comp &c) { return std::vector<int32_t>(c.dims, c.dims + c.k); }

// eq. 4.2 over the accepted set as given: b_v = sum_{u in U, u >= v} (-1)^(|u|-|v|).
// Also records whether U is downward closed (every subset of an accepted
// component accepted), which the slice-free form needs.
static int compute_b_and_check(hdmr *h) {
    std::map<std::vector<int32_t>, int> index;
    for (size_t c = 0; c < h->comps.size(); ++c) index[dims_vec(h->comps[c])] = (int)c;
    h->b.assign(h->comps.size(), 0.0);
    h->closed = true;
    for (size_t u = 0; u < h->comps.size(); ++u) {
        const Comp &cu = h->comps[u];
        for (uint32_t mask = 0; mask < (1u << cu.k); ++mask) {
            std::vector<int32_t> v;
            for (int j = 0; j < cu.k; ++j)
                if (mask & (1u << j)) v.push_back(cu.dims[j]);
            auto it = index.find(v);
            if (it == index.end()) {
                h->closed = false;
                continue;
            }
            h->b[it->second] += ((cu.k - (int)v.size()) & 1) ? -1.0 : 1.0;
        }
    }
    return DDSG_OK;
}

template <typename T>
static int dev_upload(T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return DDSG_OK;
    ALLOC_TRY(dst, sizeof(T) * src.size(), "grid tables");
    CUDA_TRY(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return DDSG_OK;
}

static int upload_tables(hdmr *h) {
    if (h->comps.empty()) return fail(DDSG_ERR_STATE, "no components");
    int rc = compute_b_and_check(h);
    if (rc) return rc;
    const int C = (int)h->comps.size();
    const int64_t P = h->P;
    if (P >= ((int64_t)1 << 31)) return fail(DDSG_ERR_TABLE, "too many points for 32-bit ids");
    std::vector<DevComp> dc(C);
    std::vector<DevTup> tups;
    std::vector<int32_t> slots;
    std::vector<int32_t> layer_pts;
    std::vector<int32_t> layer_off;
    std::vector<uint8_t> pt_lv((size_t)KMAX * P, 0);
    std::vector<uint32_t> pt_ix((size_t)KMAX * P, 0);
    std::vector<int32_t> dpos((size_t)P, -1);
    int64_t row = 0;
    bool all_tile = true;
    for (int c = 0; c < C; ++c) {
        const Comp &cp = h->comps[c];
        const int k = cp.k;
        const int64_t np = cp.npts();
        const int64_t base = h->first_point[c];
        DevComp &d = dc[c];
        memset(&d, 0, sizeof d);
        d.k = k;
        for (int j = 0; j < KMAX; ++j) d.dims[j] = cp.dims[j];
        d.pt_begin = (int32_t)base;
        d.pt_end = (int32_t)(base + np);
        d.b = h->b[c];
        for (int64_t p = 0; p < np; ++p)
            for (int j = 0; j < k; ++j) d.lmax[j] = std::max<uint8_t>(d.lmax[j], cp.lv[p * k + j]);
        if (k > 2 || d.lmax[0] > LT || d.lmax[1] > LT || h->d > 65536) all_tile = false;
        // group points by level tuple
        std::map<std::vector<uint8_t>, std::vector<int64_t>> bytup;
        for (int64_t p = 0; p < np; ++p) {
            std::vector<uint8_t> key(k);
            for (int j = 0; j < k; ++j) {
                key[j] = cp.lv[p * k + j];
                pt_lv[(size_t)j * P + base + p] = cp.lv[p * k + j];
                pt_ix[(size_t)j * P + base + p] = cp.ix[p * k + j];
            }
            bytup[key].push_back(p);
        }
        // order: (interior, level sum, lexicographic)
        std::vector<std::vector<uint8_t>> keys;
        for (auto &kv : bytup) keys.push_back(kv.first);
        auto interior = [](const std::vector<uint8_t> &t) {
            for (uint8_t l : t) if (l < 2) return 0;
            return 1;
        };
        std::stable_sort(keys.begin(), keys.end(), [&](const std::vector<uint8_t> &a, const std::vector<uint8_t> &b) {
            int ia = interior(a), ib = interior(b);
            if (ia != ib) return ia < ib;
            int sa = level_sum(a.data(), k), sb = level_sum(b.data(), k);
            if (sa != sb) return sa < sb;
            return a < b;
        });
        d.tup_begin = (int32_t)tups.size();
        d.tup_int = -1;
        for (auto &key : keys) {
            if (d.tup_int < 0 && interior(key)) d.tup_int = (int32_t)tups.size();
            DevTup t;
            memset(&t, 0, sizeof t);
            uint64_t size = 1;
            for (int j = 0; j < k; ++j) {
                t.lev[j] = key[j];
                size *= ncells(key[j]);
            }
            if (size > (1ull << 26)) return fail(DDSG_ERR_TABLE, "component %d: level tuple too fine for a dense cell directory", c);
            t.lsum = level_sum(key.data(), k);
            t.nc1 = k >= 2 ? ncells(key[1]) : 1u;
            t.first = (int32_t)row;
            // present cells of this tuple, in increasing cell index
            std::vector<std::pair<uint64_t, int64_t>> cells;
            for (int64_t p : bytup[key]) {
                uint64_t off = 0;
                for (int j = 0; j < k; ++j) off = off * ncells(key[j]) + cell_of_index(key[j], cp.ix[p * k + j]);
                cells.emplace_back(off, p);
            }
            std::sort(cells.begin(), cells.end());
            for (auto &cl : cells) dpos[base + cl.second] = (int32_t)row++;
            if (size <= 64) {
                for (auto &cl : cells) t.mask |= 1ull << cl.first;
                t.slot_base = -1;
            } else {
                if (slots.size() + size > ((size_t)1 << 31)) return fail(DDSG_ERR_TABLE, "cell directories exceed 2^31 entries");
                t.slot_base = (int32_t)slots.size();
                slots.resize(slots.size() + size, -1);
                for (auto &cl : cells) slots[t.slot_base + cl.first] = dpos[base + cl.second];
            }
            tups.push_back(t);
        }
        d.tup_end = (int32_t)tups.size();
        if (d.tup_int < 0) d.tup_int = d.tup_end;
        d.row_begin = (int32_t)(row - np);
        d.row_end = (int32_t)row;
        d.row_int = d.tup_int < d.tup_end ? tups[d.tup_int].first : d.row_end;
        // layers by level sum
        std::vector<int64_t> order(np);
        for (int64_t p = 0; p < np; ++p) order[p] = p;
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b2) {
            return level_sum(&cp.lv[a * k], k) < level_sum(&cp.lv[b2 * k], k);
        });
        d.layer_begin = (int32_t)layer_off.size();
        int maxs = k == 0 ? 0 : level_sum(&cp.lv[order[np - 1] * k], k);
        d.nlayers = maxs + 1;
        const size_t lp0 = layer_pts.size();
        size_t pos = 0;
        for (int s = 0; s <= maxs; ++s) {
            layer_off.push_back((int32_t)(lp0 + pos));
            while (pos < (size_t)np && (k == 0 ? 0 : level_sum(&cp.lv[order[pos] * k], k)) == s) {
                layer_pts.push_back((int32_t)(base + order[pos]));
                ++pos;
            }
        }
        layer_off.push_back((int32_t)(lp0 + pos));
    }
    free_tables(h->dt);
    DevTables &t = h->dt;
    t.C = C;
    t.T = (int32_t)tups.size();
    t.P = P;
    t.S = (int64_t)slots.size();
    t.m = h->m;
    t.mp64 = (h->m + 1) & ~1;
    t.mp32 = (h->m + 3) & ~3;
    t.tile_ok = all_tile ? 1 : 0;
    if ((rc = dev_upload(&t.comps, dc))) return rc;
    if ((rc = dev_upload(&t.tups, tups))) return rc;
    if ((rc = dev_upload(&t.slots, slots))) return rc;
    if ((rc = dev_upload(&t.layer_pts, layer_pts))) return rc;
    if ((rc = dev_upload(&t.layer_off, layer_off))) return rc;
    if ((rc = dev_upload(&t.pt_lv, pt_lv))) return rc;
    if ((rc = dev_upload(&t.pt_ix, pt_ix))) return rc;
    if ((rc = dev_upload(&t.pt_dpos, dpos))) return rc;
    h->dpos = dpos;
    // per-form component lists and the largest staged surplus block
    const int64_t mp64 = (h->m + 1) & ~1, mp32 = (h->m + 3) & ~3;
    for (int form = 0; form < 2; ++form) {
        h->ntup[form].resize(C);
        for (int c = 0; c < C; ++c)
            h->ntup[form][c] = dc[c].tup_end - (form == DDSG_FORM_PAPER ? dc[c].tup_begin : dc[c].tup_int);
        std::vector<int32_t> lst;
        int64_t rows_max = 0;
        for (int c = 0; c < C; ++c) {
            if (form == DDSG_FORM_PAPER && h->b[c] == 0.0) continue;
            lst.push_back(c);
            const int64_t r0 = form == DDSG_FORM_PAPER ? dc[c].row_begin : dc[c].row_int;
            rows_max = std::max<int64_t>(rows_max, dc[c].row_end - r0);
        }
        if ((rc = dev_upload(&t.proc[form], lst))) return rc;
        t.nproc[form] = (int32_t)lst.size();
        std::vector<int4> recs;
        std::vector<uint32_t> pds;
        for (int c : lst) {
            const DevComp &d = dc[c];
            const int32_t r0 = form == DDSG_FORM_PAPER ? d.row_begin : d.row_int;
            const int32_t tb = form == DDSG_FORM_PAPER ? d.tup_begin : d.tup_int;
            const uint32_t nrows = (uint32_t)(d.row_end - r0), nt = (uint32_t)(d.tup_end - tb);
            // fields fit whenever the component fits the staged kernel (rows < 2^20, tuples < 2^11)
            recs.push_back(make_int4(c, r0, (int)((nrows & 0xfffffu) | ((nt & 0x7ffu) << 20)), tb));
            const uint32_t d0 = d.k >= 1 ? (uint32_t)d.dims[0] : 0u;
            const uint32_t d1 = d.k >= 2 ? (uint32_t)d.dims[1] : d0;
            pds.push_back((d0 & 0xffffu) | (d1 << 16));
        }
        if ((rc = dev_upload(&t.stage_rec[form], recs))) return rc;
        if ((rc = dev_upload(&t.pdims[form], pds))) return rc;
        for (int c2 = 0; c2 < C; ++c2) {
            t.max_tuples = std::max(t.max_tuples, dc[c2].tup_end - dc[c2].tup_begin);
            for (int j = 0; j < dc[c2].k; ++j) t.max_level = std::max<int32_t>(t.max_level, dc[c2].lmax[j]);
        }
        t.stage_bytes[form][DDSG_F64] = rows_max * mp64 * 8;
        t.stage_bytes[form][DDSG_F32C] = rows_max * mp32 * 4;
    }
    ALLOC_TRY(&t.alpha64, sizeof(double) * (size_t)P * t.mp64, "surpluses");
    ALLOC_TRY(&t.alpha32, sizeof(float) * (size_t)P * t.mp32, "surpluses");
    CUDA_TRY(cudaMemset(t.alpha64, 0, sizeof(double) * (size_t)P * t.mp64));
    CUDA_TRY(cudaMemset(t.alpha32, 0, sizeof(float) * (size_t)P * t.mp32));
    h->uploaded = true;
    h->have_alpha = false;
    ++h->gen;
    return DDSG_OK;
}

// Nodal-slab tables of `form` for kernel 5: planned and allocated on first use
// (once per table upload), node values recomputed whenever the surpluses change.
// Tables the kernel cannot hold leave it ineligible; that is not an error.
static int ensure_nodal(hdmr *h, int form, cudaStream_t st) {
    DevNodal &N = h->dt.nod[form];
    if (!h->uploaded) return DDSG_OK;
    if (!N.tried) {
        std::vector<NodalComp> nc(h->comps.size());
        for (size_t c = 0; c < h->comps.size(); ++c) {
            const Comp &cp = h->comps[c];
            NodalComp &o = nc[c];
            o.k = cp.k;
            for (int j = 0; j < KMAX; ++j) o.dims[j] = cp.dims[j];
            o.lv = cp.lv.data();
            o.ix = cp.ix.data();
            o.npts = cp.npts();
            o.first = h->first_point[c];
            o.b = h->b[c];
        }
        const int rc = nodal_build(h->m, form, nc, h->dpos, N);
        ++h->gen;   // captured graphs hold the table pointers
        if (rc) return rc;
    }
    if (N.ok && !N.vals && h->have_alpha) {
        CUDA_TRY(launch_nodalize(N, h->dt.alpha64, h->dt.mp64, h->m, st));
        N.vals = 1;
    }
    return DDSG_OK;
}

extern "C" int hdmr_hierarchize(hdmr_t *h, const double *values_dev, ddsg_stream_t stream) {
    if (!h || !values_dev) return fail(DDSG_ERR_ARG, "hdmr_hierarchize: NULL argument");
    if (int rc0 = ensure_device(h)) return rc0;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DDSG_ERR_CUDA, "hdmr_hierarchize: cannot select device");
    if (!h->uploaded) {
        int rc = upload_tables(h);
        if (rc) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    {
        ProfScope ps(h, DDSG_K_HIER, st);
        CUDA_TRY(launch_hierarchize(h->dt, h->m, values_dev, st));
    }
    {
        ProfScope ps(h, DDSG_K_CONVERT, st);
        CUDA_TRY(launch_to_f32(h->dt.alpha64, h->dt.mp64, h->dt.alpha32, h->dt.mp32, h->P, h->m, st));
    }
    h->have_alpha = true;
    for (int form = 0; form < 2; ++form) {
        DevNodal &N = h->dt.nod[form];
        N.vals = 0;
        if (N.ok) {
            ProfScope ps(h, DDSG_K_CONVERT, st);
            CUDA_TRY(launch_nodalize(N, h->dt.alpha64, h->dt.mp64, h->m, st));
            N.vals = 1;
        }
    }
    return DDSG_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / resume: one binary file per expansion
//   "DDSGHDMR", u32 version (1), u32 0, i32 d, m, order, ncomp, i64 P,
//   f64 anchor[d], lo[d], hi[d],
//   per component: i32 k, i32 dims[k], i64 npts, u8 levels[npts*k], u32 indices[npts*k],
//   f64 surpluses[P*m] (points in component / table order),
//   u64 FNV-1a of every byte after the 16-byte header.
// ---------------------------------------------------------------------------

namespace {

constexpr char kMagic[8] = {'D', 'D', 'S', 'G', 'H', 'D', 'M', 'R'};
constexpr uint32_t kFileVersion = 1;

using io::Reader;
using io::Writer;

}  // namespace

extern "C" int hdmr_save(const hdmr_t *h, const char *path) {
    if (!h || !path) return fail(DDSG_ERR_ARG, "hdmr_save: NULL argument");
    if (!h->have_alpha) return fail(DDSG_ERR_STATE, "hdmr_save: hierarchize first");
    std::vector<double> alpha((size_t)h->P * h->m);
    int rc = hdmr_get_surpluses(h, alpha.data(), nullptr);
    if (rc) return rc;
    Writer w;
    w.header(kMagic, kFileVersion);
    w.put1<int32_t>(h->d);
    w.put1<int32_t>(h->m);
    w.put1<int32_t>(h->order);
    w.put1<int32_t>((int32_t)h->comps.size());
    w.put1<int64_t>(h->P);
    w.put(h->anchor.data(), h->d);
    w.put(h->lo.data(), h->d);
    w.put(h->hi.data(), h->d);
    for (const Comp &c : h->comps) {
        w.put1<int32_t>(c.k);
        w.put(c.dims, c.k);
        w.put1<int64_t>(c.npts());
        if (c.k) {
            w.put(c.lv.data(), c.lv.size());
            w.put(c.ix.data(), c.ix.size());
        }
    }
    w.put(alpha.data(), alpha.size());
    w.seal();
    if (!io::write_file(path, w.buf)) return fail(DDSG_ERR_ARG, "hdmr_save: write to %s failed", path);
    return DDSG_OK;
}

extern "C" int hdmr_load(const char *path, hdmr_t **out) {
    if (!path || !out) return fail(DDSG_ERR_ARG, "hdmr_load: NULL argument");
    *out = nullptr;
    std::vector<unsigned char> buf;
    if (!io::read_file(path, buf)) return fail(DDSG_ERR_ARG, "hdmr_load: cannot open %s", path);
    Reader r{nullptr, nullptr};
    uint32_t version = 0;
    switch (io::open_body(buf, kMagic, kFileVersion, r, &version)) {
        case 1: return fail(DDSG_ERR_ARG, "hdmr_load: %s is not an expansion file", path);
        case 2: return fail(DDSG_ERR_ARG, "hdmr_load: unsupported file version %u", version);
        case 3: return fail(DDSG_ERR_ARG, "hdmr_load: checksum mismatch (truncated or corrupt file)");
        default: break;
    }
    int32_t d = 0, m = 0, order = 0, nc = 0;
    int64_t P = 0;
    r.get(&d, 1);
    r.get(&m, 1);
    r.get(&order, 1);
    r.get(&nc, 1);
    r.get(&P, 1);
    if (!r.ok || d < 1 || m < 1 || nc < 0 || P < 0 || (size_t)d > buf.size() || (size_t)nc > buf.size())
        return fail(DDSG_ERR_ARG, "hdmr_load: bad header");
    std::vector<double> anchor(d), lo(d), hi(d);
    r.get(anchor.data(), d);
    r.get(lo.data(), d);
    r.get(hi.data(), d);
    if (!r.ok) return fail(DDSG_ERR_ARG, "hdmr_load: truncated header");
    hdmr_t *h = nullptr;
    int rc = hdmr_create(d, m, order, anchor.data(), lo.data(), hi.data(), &h);
    if (rc) return rc;
    for (int32_t c = 0; c < nc; ++c) {
        int32_t kk = -1, dims[KMAX];
        int64_t npts = -1;
        r.get(&kk, 1);
        if (!r.ok || kk < 0 || kk > KMAX) {
            hdmr_destroy(h);
            return fail(DDSG_ERR_ARG, "hdmr_load: bad component record %d", c);
        }
        r.get(dims, kk);
        r.get(&npts, 1);
        if (!r.ok || npts < 0 || (size_t)npts > buf.size()) {
            hdmr_destroy(h);
            return fail(DDSG_ERR_ARG, "hdmr_load: bad component record %d", c);
        }
        std::vector<uint8_t> lv((size_t)npts * kk);
        std::vector<uint32_t> ix((size_t)npts * kk);
        r.get(lv.data(), lv.size());
        r.get(ix.data(), ix.size());
        if (!r.ok) {
            hdmr_destroy(h);
            return fail(DDSG_ERR_ARG, "hdmr_load: truncated component %d", c);
        }
        int32_t cid = 0;
        if ((rc = hdmr_add_component(h, kk, dims, npts, kk ? lv.data() : nullptr, kk ? ix.data() : nullptr, &cid))) {
            hdmr_destroy(h);
            return rc;
        }
    }
    if (h->P != P) {
        hdmr_destroy(h);
        return fail(DDSG_ERR_ARG, "hdmr_load: point count mismatch");
    }
    std::vector<double> alpha((size_t)P * m);
    r.get(alpha.data(), alpha.size());
    if (!r.ok || r.p != r.end) {
        hdmr_destroy(h);
        return fail(DDSG_ERR_ARG, "hdmr_load: surplus block has the wrong size");
    }
    // install the surpluses in device-row order (FP64, then the FP32 copy)
    if ((rc = ensure_device(h))) {
        hdmr_destroy(h);
        return rc;
    }
    {
        DeviceGuard g(h->device);
        if (!h->uploaded && (rc = upload_tables(h))) {
            hdmr_destroy(h);
            return rc;
        }
        const int mp = h->dt.mp64;
        std::vector<double> dev((size_t)P * mp, 0.0);
        for (int64_t p = 0; p < P; ++p)
            std::copy(&alpha[(size_t)p * m], &alpha[(size_t)p * m] + m, &dev[(size_t)h->dpos[p] * mp]);
        if (cudaMemcpy(h->dt.alpha64, dev.data(), sizeof(double) * dev.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            launch_to_f32(h->dt.alpha64, h->dt.mp64, h->dt.alpha32, h->dt.mp32, h->P, h->m, nullptr) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess) {
            cudaGetLastError();
            hdmr_destroy(h);
            return fail(DDSG_ERR_CUDA, "hdmr_load: surplus upload failed");
        }
        h->have_alpha = true;
    }
    *out = h;
    return DDSG_OK;
}

extern "C" int hdmr_shape(const hdmr_t *h, int32_t *d, int32_t *m, int32_t *order, double *anchor_host,
                          double *lo_host, double *hi_host) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_shape: NULL handle");
    if (d) *d = h->d;
    if (m) *m = h->m;
    if (order) *order = h->order;
    if (anchor_host) std::copy(h->anchor.begin(), h->anchor.end(), anchor_host);
    if (lo_host) std::copy(h->lo.begin(), h->lo.end(), lo_host);
    if (hi_host) std::copy(h->hi.begin(), h->hi.end(), hi_host);
    return DDSG_OK;
}

extern "C" int hdmr_quadrature(hdmr_t *h, double *q_dev, ddsg_stream_t stream) {
    if (!h || !q_dev) return fail(DDSG_ERR_ARG, "hdmr_quadrature: NULL argument");
    if (!h->uploaded || !h->have_alpha) return fail(DDSG_ERR_STATE, "hdmr_quadrature: call hdmr_hierarchize first");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DDSG_ERR_CUDA, "hdmr_quadrature: cannot select device");
    CUDA_TRY(launch_quadrature(h->dt, h->m, q_dev, reinterpret_cast<cudaStream_t>(stream)));
    return DDSG_OK;
}

// Expansion and active-dimension criteria of Alg. 2 from the component
// integrals (eq. 3.7): the cut-HDMR component integrals by inclusion-exclusion
// over the subsets of each component (every subset must be a component),
// eta_u (eq. 3.19) for the components of order k and rho (eq. 3.18).
extern "C" int hdmr_expansion_norms(hdmr_t *h, int k, double eps_eta, double *qf_host, double *eta_host,
                                    double *rho_all, double *rho_kept, ddsg_stream_t stream) {
    if (!h || k < 1) return fail(DDSG_ERR_ARG, "hdmr_expansion_norms: bad argument");
    if (!h->uploaded || !h->have_alpha) return fail(DDSG_ERR_STATE, "hdmr_expansion_norms: call hdmr_hierarchize first");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DDSG_ERR_CUDA, "hdmr_expansion_norms: cannot select device");
    const int C = (int)h->comps.size(), m = h->m;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double *qd = nullptr;
    ALLOC_TRY(&qd, sizeof(double) * (size_t)C * m, "hdmr_expansion_norms");
    std::vector<double> Q((size_t)C * m);
    cudaError_t e = launch_quadrature(h->dt, m, qd, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Q.data(), qd, sizeof(double) * Q.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(qd);
    if (e != cudaSuccess) return fail(DDSG_ERR_CUDA, "hdmr_expansion_norms: %s", cudaGetErrorString(e));
    // component index by dimension set
    std::map<std::vector<int32_t>, int> index;
    for (int c = 0; c < C; ++c) index[std::vector<int32_t>(h->comps[c].dims, h->comps[c].dims + h->comps[c].k)] = c;
    std::vector<double> Qf((size_t)C * m, 0.0);
    for (int c = 0; c < C; ++c) {
        const int kc = h->comps[c].k;
        for (uint32_t mask = 0; mask < (1u << kc); ++mask) {
            std::vector<int32_t> v;
            for (int j = 0; j < kc; ++j)
                if (mask >> j & 1u) v.push_back(h->comps[c].dims[j]);
            auto it = index.find(v);
            if (it == index.end()) return fail(DDSG_ERR_ARG, "hdmr_expansion_norms: component %d lacks a subset component", c);
            const double sign = ((kc - (int)v.size()) & 1) ? -1.0 : 1.0;
            for (int o = 0; o < m; ++o) Qf[(size_t)c * m + o] += sign * Q[(size_t)it->second * m + o];
        }
    }
    std::vector<double> lower(m, 0.0), num_all(m, 0.0), num_kept(m, 0.0);
    for (int c = 0; c < C; ++c)
        if (h->comps[c].k <= k - 1)
            for (int o = 0; o < m; ++o) lower[o] += Qf[(size_t)c * m + o];
    auto norm = [m](const double *v) {
        double s = 0.0;
        for (int o = 0; o < m; ++o) s += v[o] * v[o];
        return sqrt(s);
    };
    const double nl = norm(lower.data());
    for (int c = 0; c < C; ++c) {
        double eta = NAN;
        if (h->comps[c].k == k) {
            eta = norm(&Qf[(size_t)c * m]) / nl;
            for (int o = 0; o < m; ++o) num_all[o] += Qf[(size_t)c * m + o];
            if (k < 2 || eta > eps_eta)
                for (int o = 0; o < m; ++o) num_kept[o] += Qf[(size_t)c * m + o];
        }
        if (eta_host) eta_host[c] = eta;
    }
    if (qf_host) std::copy(Qf.begin(), Qf.end(), qf_host);
    if (rho_all) *rho_all = norm(num_all.data()) / nl;
    if (rho_kept) *rho_kept = norm(num_kept.data()) / nl;
    return DDSG_OK;
}

extern "C" int hdmr_get_surpluses(const hdmr_t *h, double *alpha_host, ddsg_stream_t stream) {
    if (!h || !alpha_host) return fail(DDSG_ERR_ARG, "hdmr_get_surpluses: NULL argument");
    if (!h->have_alpha) return fail(DDSG_ERR_STATE, "hdmr_get_surpluses: not hierarchized");
    DeviceGuard g(h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int mp = h->dt.mp64, m = h->m;
    std::vector<double> tmp((size_t)h->P * mp);
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), h->dt.alpha64, sizeof(double) * tmp.size(),
                             cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t p = 0; p < h->P; ++p)
        std::copy(&tmp[(size_t)h->dpos[p] * mp], &tmp[(size_t)h->dpos[p] * mp] + m, alpha_host + p * m);
    return DDSG_OK;
}

extern "C" int hdmr_get_b(const hdmr_t *h, double *b_host) {
    if (!h || !b_host) return fail(DDSG_ERR_ARG, "hdmr_get_b: NULL argument");
    if (!h->uploaded) {
        int rc = compute_b_and_check(const_cast<hdmr *>(h));
        if (rc) return rc;
    }
    std::copy(h->b.begin(), h->b.end(), b_host);
    return DDSG_OK;
}

// ---------------------------------------------------------------------------
// refinement (eq. 3.8)
// ---------------------------------------------------------------------------

static int children1d(int l, uint32_t i, uint32_t *ci) {
    if (l == 1) { ci[0] = 0; ci[1] = 2; return 2; }
    if (l == 2) { ci[0] = i == 0 ? 1u : 3u; return 1; }
    ci[0] = 2 * i - 1;
    ci[1] = 2 * i + 1;
    return 2;
}

static void parent1d(int l, uint32_t i, int *pl, uint32_t *pi) {
    if (l == 2) { *pl = 1; *pi = 1; return; }
    if (l == 3) { *pl = 2; *pi = i == 1 ? 0u : 2u; return; }
    *pl = l - 1;
    const uint32_t a = (i - 1) / 2, b = (i + 1) / 2;
    *pi = (a & 1u) ? a : b;
}

extern "C" int hdmr_refine(hdmr_t *h, double eps, int max_level, int strict, int64_t *n_new,
                           ddsg_stream_t stream) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_refine: NULL handle");
    if (max_level < 1 || max_level > LMAX) return fail(DDSG_ERR_ARG, "hdmr_refine: max_level out of range");
    if (!h->have_alpha) return fail(DDSG_ERR_STATE, "hdmr_refine: surpluses not computed");
    const int m = h->m;
    std::vector<double> alpha((size_t)h->P * m);
    int rc = hdmr_get_surpluses(h, alpha.data(), stream);
    if (rc) return rc;
    // eq. 3.8 compares |alpha| with eps; a non-finite surplus (from a non-finite
    // value handed to hdmr_hierarchize) would silently read as insignificant
    for (size_t c = 0; c < h->comps.size(); ++c) {
        const int64_t np = h->comps[c].npts();
        const double *al = alpha.data() + (size_t)h->first_point[c] * m;
        for (int64_t q = 0; q < np * m; ++q)
            if (!std::isfinite(al[q]))
                return fail(DDSG_ERR_NUMERIC, "hdmr_refine: surplus of component %zu, point %lld, output %d is not finite",
                            c, (long long)(q / m), (int)(q % m));
    }
    int64_t added = 0;
    for (size_t c = 0; c < h->comps.size(); ++c) {
        Comp &cp = h->comps[c];
        const int k = cp.k;
        if (k == 0) continue;
        const int64_t np = cp.npts();
        const double *al = alpha.data() + (size_t)h->first_point[c] * m;
        std::unordered_map<std::string, int64_t> present;
        present.reserve((size_t)np * 2);
        for (int64_t p = 0; p < np; ++p) present.emplace(point_key(&cp.lv[p * k], &cp.ix[p * k], k), p);
        auto significant = [&](int64_t p) {
            double g = 0.0;
            for (int j = 0; j < m; ++j) g = std::max(g, fabs(al[p * m + j]));
            return g > eps;
        };
        struct Cand { uint8_t lv[KMAX]; uint32_t ix[KMAX]; };
        std::vector<Cand> cand;
        std::unordered_map<std::string, int> seen;
        for (int64_t p = 0; p < np; ++p) {
            if (!significant(p)) continue;
            for (int j = 0; j < k; ++j) {
                uint32_t ci[2];
                const int nch = children1d(cp.lv[p * k + j], cp.ix[p * k + j], ci);
                for (int q = 0; q < nch; ++q) {
                    Cand o;
                    memset(&o, 0, sizeof o);
                    for (int r = 0; r < k; ++r) {
                        o.lv[r] = cp.lv[p * k + r];
                        o.ix[r] = cp.ix[p * k + r];
                    }
                    o.lv[j] = (uint8_t)(o.lv[j] + 1);
                    o.ix[j] = ci[q];
                    if (o.lv[j] > LMAX || level_sum(o.lv, k) > max_level - 1) continue;
                    const std::string key = point_key(o.lv, o.ix, k);
                    if (present.count(key) || seen.count(key)) continue;
                    if (strict) {
                        bool ok = true;
                        for (int r = 0; r < k && ok; ++r) {
                            if (o.lv[r] < 2) continue;
                            Cand par = o;
                            int pl;
                            uint32_t pi;
                            parent1d(o.lv[r], o.ix[r], &pl, &pi);
                            par.lv[r] = (uint8_t)pl;
                            par.ix[r] = pi;
                            auto it = present.find(point_key(par.lv, par.ix, k));
                            if (it != present.end() && !significant(it->second)) ok = false;
                        }
                        if (!ok) continue;
                    }
                    seen.emplace(key, 1);
                    cand.push_back(o);
                }
            }
        }
        std::sort(cand.begin(), cand.end(), [k](const Cand &a, const Cand &b) {
            const int sa = level_sum(a.lv, k), sb = level_sum(b.lv, k);
            if (sa != sb) return sa < sb;
            for (int j = 0; j < k; ++j) if (a.lv[j] != b.lv[j]) return a.lv[j] < b.lv[j];
            for (int j = 0; j < k; ++j) if (a.ix[j] != b.ix[j]) return a.ix[j] < b.ix[j];
            return false;
        });
        for (const Cand &o : cand) {
            cp.lv.insert(cp.lv.end(), o.lv, o.lv + k);
            cp.ix.insert(cp.ix.end(), o.ix, o.ix + k);
        }
        added += (int64_t)cand.size();
    }
    if (added) {
        rebuild_offsets(h);
        h->uploaded = false;
        h->have_alpha = false;
    }
    if (n_new) *n_new = added;
    return DDSG_OK;
}

// ---------------------------------------------------------------------------
// evaluation
// ---------------------------------------------------------------------------

static int ensure_ws(hdmr *h, int64_t n) {
    const size_t need = (size_t)n * h->d * sizeof(uint64_t) + (size_t)n * sizeof(int32_t) + 256;
    if (need <= h->ws_bytes) return DDSG_OK;
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
    ++h->gen;
    if (dev_alloc(&h->ws, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(DDSG_ERR_OOM, "hdmr_eval: workspace of %zu bytes unavailable", need);
    }
    h->ws_bytes = need;
    return DDSG_OK;
}

extern "C" int hdmr_reserve(hdmr_t *h, int64_t n) {
    if (!h || n < 0) return fail(DDSG_ERR_ARG, "hdmr_reserve: bad argument");
    if (int rc0 = ensure_device(h)) return rc0;
    DeviceGuard g(h->device);
    return ensure_ws(h, n);
}

extern "C" int hdmr_eval(hdmr_t *h, int64_t n, const double *x_dev, double *y_dev, int precision,
                         int form, uint64_t *hash_dev, int32_t *count_dev, ddsg_stream_t stream) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_eval: NULL handle");
    if (n < 0) return fail(DDSG_ERR_ARG, "hdmr_eval: n < 0");
    if (n == 0) return DDSG_OK;
    if (!x_dev || !y_dev) return fail(DDSG_ERR_ARG, "hdmr_eval: NULL x or y");
    if (precision != DDSG_F64 && precision != DDSG_F32C) return fail(DDSG_ERR_ARG, "hdmr_eval: unknown precision %d", precision);
    if (form != DDSG_FORM_PAPER && form != DDSG_FORM_SLICEFREE) return fail(DDSG_ERR_ARG, "hdmr_eval: unknown form %d", form);
    if (!h->uploaded || !h->have_alpha) return fail(DDSG_ERR_STATE, "hdmr_eval: call hdmr_hierarchize first");
    if (form == DDSG_FORM_SLICEFREE && !h->anchor_central)
        return fail(DDSG_ERR_ARG, "hdmr_eval: the slice-free form needs the anchor at the domain centre");
    if (form == DDSG_FORM_SLICEFREE && !h->closed)
        return fail(DDSG_ERR_ARG, "hdmr_eval: the slice-free form needs a downward-closed component set");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DDSG_ERR_CUDA, "hdmr_eval: cannot select device");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (kernel_is_nodal(h->cfg[precision][form].kernel) && !h->capturing) {
        if (int rc0 = ensure_nodal(h, form, st)) return rc0;
    }
    if (!eval_kernel_eligible(h->dt, h->cfg[precision][form].kernel, precision, form))
        h->cfg[precision][form] = EvalConfig();
    int rc = ensure_ws(h, n);
    if (rc) return rc;
    uint64_t *X = reinterpret_cast<uint64_t *>(h->ws);
    {
        ProfScope ps(h, DDSG_K_ENCODE, st);
        CUDA_TRY(launch_encode_queries(n, h->d, x_dev, h->dlo, h->dspan, X, h->stats, st));
    }
    EvalArgs a;
    a.t = &h->dt;
    a.d = h->d;
    a.m = h->m;
    a.n = n;
    a.X = X;
    a.y = y_dev;
    a.hash = hash_dev;
    a.count = count_dev;
    a.form = form;
    a.precision = precision;
    a.cfg = h->cfg[precision][form];
    a.err = reinterpret_cast<unsigned long long *>(h->stats + 2);
    a.withhold_from = h->fi_withhold;
    {
        ProfScope ps(h, DDSG_K_EVAL, st);
        CUDA_TRY(launch_eval(a, st));
    }
    return DDSG_OK;
}

extern "C" int hdmr_set_fault_injection(hdmr_t *h, int withhold_from) {
    if (!h || withhold_from < -1) return fail(DDSG_ERR_ARG, "hdmr_set_fault_injection: bad argument");
    h->fi_withhold = withhold_from;
    ++h->gen;
    return DDSG_OK;
}

extern "C" int hdmr_eval_graph(hdmr_t *h, int64_t n, const double *x_dev, double *y_dev, int precision,
                               int form, ddsg_stream_t stream) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_eval_graph: NULL handle");
    if (n < 0) return fail(DDSG_ERR_ARG, "hdmr_eval_graph: n < 0");
    if (n == 0) return DDSG_OK;
    if (!x_dev || !y_dev) return fail(DDSG_ERR_ARG, "hdmr_eval_graph: NULL x or y");
    if (precision != DDSG_F64 && precision != DDSG_F32C)
        return fail(DDSG_ERR_ARG, "hdmr_eval_graph: unknown precision %d", precision);
    if (form != DDSG_FORM_PAPER && form != DDSG_FORM_SLICEFREE)
        return fail(DDSG_ERR_ARG, "hdmr_eval_graph: unknown form %d", form);
    if (!h->uploaded || !h->have_alpha) return fail(DDSG_ERR_STATE, "hdmr_eval_graph: call hdmr_hierarchize first");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(DDSG_ERR_CUDA, "hdmr_eval_graph: cannot select device");
    if (kernel_is_nodal(h->cfg[precision][form].kernel)) {   // any allocation happens before the capture
        if (int rc0 = ensure_nodal(h, form, reinterpret_cast<cudaStream_t>(stream))) return rc0;
    }
    if (!eval_kernel_eligible(h->dt, h->cfg[precision][form].kernel, precision, form))
        h->cfg[precision][form] = EvalConfig();
    int rc = ensure_ws(h, n);   // any allocation happens before the capture
    if (rc) return rc;
    if (!h->gstream) {
        CUDA_TRY(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
        for (auto &e : h->gev) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const EvalConfig cfg = h->cfg[precision][form];
    const bool hit = h->gexec && h->g_n == n && h->g_x == x_dev && h->g_y == y_dev && h->g_prec == precision &&
                     h->g_form == form && h->g_cfg.kernel == cfg.kernel && h->g_cfg.mc == cfg.mc &&
                     h->g_gen == h->gen;
    if (!hit) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        CUDA_TRY(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeRelaxed));
        h->capturing = true;
        rc = hdmr_eval(h, n, x_dev, y_dev, precision, form, nullptr, nullptr,
                       reinterpret_cast<ddsg_stream_t>(h->gstream));
        h->capturing = false;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(h->gstream, &graph);
        if (rc || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc ? rc : fail(DDSG_ERR_CUDA, "hdmr_eval_graph: capture failed: %s", cudaGetErrorString(ec));
        }
        const cudaError_t ei = cudaGraphInstantiate(&h->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            h->gexec = nullptr;
            cudaGetLastError();
            return fail(DDSG_ERR_CUDA, "hdmr_eval_graph: instantiate failed: %s", cudaGetErrorString(ei));
        }
        h->g_n = n;
        h->g_x = x_dev;
        h->g_y = y_dev;
        h->g_prec = precision;
        h->g_form = form;
        h->g_cfg = cfg;
        h->g_gen = h->gen;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaEventRecord(h->gev[0], st));
    CUDA_TRY(cudaStreamWaitEvent(h->gstream, h->gev[0], 0));
    {
        ProfScope ps(h, DDSG_K_GRAPH, h->gstream);
        CUDA_TRY(cudaGraphLaunch(h->gexec, h->gstream));
    }
    CUDA_TRY(cudaEventRecord(h->gev[1], h->gstream));
    CUDA_TRY(cudaStreamWaitEvent(st, h->gev[1], 0));
    return DDSG_OK;
}

extern "C" int hdmr_eval_host(hdmr_t *h, int64_t n, const double *x_host, double *y_host,
                              int precision, int form, ddsg_stream_t stream) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_eval_host: NULL handle");
    if (n < 0) return fail(DDSG_ERR_ARG, "hdmr_eval_host: n < 0");
    if (n == 0) return DDSG_OK;
    if (!x_host || !y_host) return fail(DDSG_ERR_ARG, "hdmr_eval_host: NULL x or y");
    if (!h->uploaded || !h->have_alpha) return fail(DDSG_ERR_STATE, "hdmr_eval_host: call hdmr_hierarchize first");
    DeviceGuard g(h->device);
    // Page-locked (pinned) queries are read by the encoding kernel straight from
    // host memory through their mapped device address: the transfer overlaps the
    // encoding instead of preceding it. Other host memory is copied first.
    auto mapped = [](const void *p) -> void * {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, p) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            return pa.devicePointer;
        cudaGetLastError();
        return nullptr;
    };
    const double *x_mapped = static_cast<const double *>(mapped(x_host));
    double *y_mapped = static_cast<double *>(mapped(y_host));
    const size_t xb = sizeof(double) * (size_t)n * h->d, yb = sizeof(double) * (size_t)n * h->m;
    const size_t need = (x_mapped ? 0 : xb) + (y_mapped ? 0 : yb) + 256;
    if (need > h->hbuf_bytes) {
        cudaFree(h->hbuf);
        h->hbuf = nullptr;
        h->hbuf_bytes = 0;
        if (dev_alloc(&h->hbuf, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(DDSG_ERR_OOM, "hdmr_eval_host: staging buffer of %zu bytes unavailable", need);
        }
        h->hbuf_bytes = need;
    }
    double *yd = reinterpret_cast<double *>(h->hbuf);
    double *xd = yd + (y_mapped ? 0 : (size_t)n * h->m);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!x_mapped) {
        ProfScope ps(h, DDSG_K_COPY, st);
        CUDA_TRY(cudaMemcpyAsync(xd, x_host, xb, cudaMemcpyHostToDevice, st));
    }
    int rc = hdmr_eval(h, n, x_mapped ? x_mapped : xd, y_mapped ? y_mapped : yd, precision, form, nullptr,
                       nullptr, stream);
    if (rc) return rc;
    if (!y_mapped) {
        ProfScope ps(h, DDSG_K_COPY, st);
        CUDA_TRY(cudaMemcpyAsync(y_host, yd, yb, cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    return DDSG_OK;
}

extern "C" int hdmr_set_eval_config(hdmr_t *h, int precision, int form, int kernel, int mc) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_set_eval_config: NULL handle");
    if (precision < 0 || precision > 1 || form < 0 || form > 1 || kernel < 0 || kernel >= NKERNELS)
        return fail(DDSG_ERR_ARG, "hdmr_set_eval_config: bad precision/form/kernel");
    if (kernel_is_nodal(kernel) && h->uploaded && h->device >= 0) {
        DeviceGuard g(h->device);
        if (int rc0 = ensure_nodal(h, form, nullptr)) return rc0;
        if (h->have_alpha && cudaDeviceSynchronize() != cudaSuccess) {
            cudaGetLastError();
            return fail(DDSG_ERR_CUDA, "hdmr_set_eval_config: computing the node values failed");
        }
    }
    if (h->uploaded && h->have_alpha && !eval_kernel_eligible(h->dt, kernel, precision, form))
        return fail(DDSG_ERR_ARG, "hdmr_set_eval_config: kernel %d cannot run these tables (a component's staged block exceeds the staging buffer)", kernel);
    int cand[16];
    const int nc = eval_mc_candidates(precision, kernel, cand, 16);
    bool ok = mc == 0;
    for (int i = 0; i < nc; ++i) ok = ok || cand[i] == mc;
    if (!ok) return fail(DDSG_ERR_ARG, "hdmr_set_eval_config: output chunk %d not compiled", mc);
    h->cfg[precision][form].kernel = kernel;
    h->cfg[precision][form].mc = mc;
    return DDSG_OK;
}

extern "C" int hdmr_nodal_info(hdmr_t *h, int form, int32_t *eligible, int64_t *rows, double *rows_per_query) {
    if (!h || form < 0 || form > 1) return fail(DDSG_ERR_ARG, "hdmr_nodal_info: bad argument");
    if (!h->uploaded || h->device < 0) return fail(DDSG_ERR_STATE, "hdmr_nodal_info: call hdmr_hierarchize first");
    DeviceGuard g(h->device);
    if (int rc0 = ensure_nodal(h, form, nullptr)) return rc0;
    const DevNodal &N = h->dt.nod[form];
    if (eligible) *eligible = N.ok ? 1 : 0;
    if (rows) *rows = N.rows;
    if (rows_per_query) *rows_per_query = N.erows;
    return DDSG_OK;
}

extern "C" int hdmr_get_eval_config(const hdmr_t *h, int precision, int form, int *kernel, int *mc) {
    if (!h || precision < 0 || precision > 1 || form < 0 || form > 1)
        return fail(DDSG_ERR_ARG, "hdmr_get_eval_config: bad argument");
    if (kernel) *kernel = h->cfg[precision][form].kernel;
    if (mc) *mc = h->cfg[precision][form].mc;
    return DDSG_OK;
}

// Times every compiled (kernel, output chunk) pair on the caller's queries
// and keeps the fastest for this precision and form.
extern "C" int hdmr_autotune(hdmr_t *h, int64_t n, const double *x_dev, double *y_dev, int precision,
                             int form, ddsg_stream_t stream, double *best_ms) {
    if (!h || n <= 0 || !x_dev || !y_dev) return fail(DDSG_ERR_ARG, "hdmr_autotune: bad argument");
    if (precision < 0 || precision > 1 || form < 0 || form > 1) return fail(DDSG_ERR_ARG, "hdmr_autotune: bad precision/form");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool prof = h->prof;
    h->prof = false;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    EvalConfig best;
    double best_t = 1e300;
    for (int kernel = 0; kernel < NKERNELS; ++kernel) {
        if (kernel_is_nodal(kernel)) {
            const int rc0 = ensure_nodal(h, form, st);
            if (rc0) { h->prof = prof; return rc0; }
        }
        if (!eval_kernel_eligible(h->dt, kernel, precision, form)) continue;
        int cand[16];
        const int nc = eval_mc_candidates(precision, kernel, cand, 16);
        for (int i = 0; i < nc; ++i) {
            h->cfg[precision][form].kernel = kernel;
            h->cfg[precision][form].mc = cand[i];
            int rc = hdmr_eval(h, n, x_dev, y_dev, precision, form, nullptr, nullptr, stream);
            if (rc) { h->prof = prof; return rc; }
            double t = 0.0;
            for (int rep = 0; rep < 2; ++rep) {
                CUDA_TRY(cudaEventRecord(e0, st));
                rc = hdmr_eval(h, n, x_dev, y_dev, precision, form, nullptr, nullptr, stream);
                if (rc) { h->prof = prof; return rc; }
                CUDA_TRY(cudaEventRecord(e1, st));
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                t = rep == 0 ? ms : std::min(t, (double)ms);
            }
            if (t < best_t) {
                best_t = t;
                best.kernel = kernel;
                best.mc = cand[i];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cfg[precision][form] = best;
    h->prof = prof;
    if (best_ms) *best_ms = best_t;
    return DDSG_OK;
}

extern "C" int hdmr_profile(hdmr_t *h, int enable) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_profile: NULL handle");
    h->prof = enable != 0;
    return DDSG_OK;
}

extern "C" int hdmr_profile_read(hdmr_t *h, double *ms, int64_t *launches, int reset) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_profile_read: NULL handle");
    if (h->device >= 0) {
        DeviceGuard g(h->device);
        for (auto &r : h->recs) {
            CUDA_TRY(cudaEventSynchronize(r.b));
            float t = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
            h->prof_ms[r.kind] += t;
            h->prof_n[r.kind] += 1;
            h->pool.push_back(r.a);
            h->pool.push_back(r.b);
        }
        h->recs.clear();
    }
    for (int k = 0; k < DDSG_NKINDS; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (launches) launches[k] = h->prof_n[k];
        if (reset) { h->prof_ms[k] = 0; h->prof_n[k] = 0; }
    }
    return DDSG_OK;
}

extern "C" int hdmr_stats(hdmr_t *h, int64_t *stats_host, int reset, ddsg_stream_t stream) {
    if (!h || !stats_host) return fail(DDSG_ERR_ARG, "hdmr_stats: NULL argument");
    if (int rc0 = ensure_device(h)) return rc0;
    DeviceGuard g(h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemcpyAsync(stats_host, h->stats, sizeof(int64_t) * 3, cudaMemcpyDeviceToHost, st));
    if (reset) CUDA_TRY(cudaMemsetAsync(h->stats, 0, sizeof(int64_t) * 4, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return DDSG_OK;
}

extern "C" int hdmr_check(hdmr_t *h, ddsg_stream_t stream) {
    if (!h) return fail(DDSG_ERR_ARG, "hdmr_check: NULL handle");
    if (h->device < 0) return DDSG_OK;   // nothing ran yet
    DeviceGuard g(h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int64_t timeouts = 0;
    CUDA_TRY(cudaMemcpyAsync(&timeouts, h->stats + 2, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (timeouts > 0) {
        CUDA_TRY(cudaMemsetAsync(h->stats + 2, 0, sizeof(int64_t), st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return fail(DDSG_ERR_TIMEOUT, "%lld warps of the staged evaluation gave up a bounded wait; their queries read NaN",
                    (long long)timeouts);
    }
#if defined(DDSG_CHECKED)
    const uint64_t w = check_word_take_kernels() | check_word_take_irbc();
    if (w) {
        std::string sites;
        for (int s = 0; s < CK_NSITES; ++s)
            if (w >> s & 1) sites += std::string(sites.empty() ? "" : ", ") + kCheckSiteName[s];
        return fail(DDSG_ERR_TABLE, "checked build: table index tests failed at: %s", sites.c_str());
    }
#endif
    return DDSG_OK;
}

// ---------------------------------------------------------------------------
// read-only view of a ready handle for entry points in other translation units
// ---------------------------------------------------------------------------

namespace ddsg {
int handle_comp_tuples(hdmr_t *h, int form, std::vector<int32_t> &out) {
    if (!h || form < 0 || form > 1) return fail(DDSG_ERR_ARG, "NULL handle or unknown form");
    if (!h->uploaded || h->ntup[form].size() != h->comps.size()) return fail(DDSG_ERR_STATE, "call hdmr_hierarchize first");
    out = h->ntup[form];
    return DDSG_OK;
}

int handle_eval_view(hdmr_t *h, int precision, int form, HandleView *v) {
    if (!h || !v) return fail(DDSG_ERR_ARG, "NULL handle");
    if (precision != DDSG_F64 && precision != DDSG_F32C) return fail(DDSG_ERR_ARG, "unknown precision %d", precision);
    if (form != DDSG_FORM_PAPER && form != DDSG_FORM_SLICEFREE) return fail(DDSG_ERR_ARG, "unknown form %d", form);
    if (!h->uploaded || !h->have_alpha || h->device < 0)
        return fail(DDSG_ERR_STATE, "call hdmr_hierarchize first");
    if (form == DDSG_FORM_SLICEFREE && !h->anchor_central)
        return fail(DDSG_ERR_ARG, "the slice-free form needs the anchor at the domain centre");
    if (form == DDSG_FORM_SLICEFREE && !h->closed)
        return fail(DDSG_ERR_ARG, "the slice-free form needs a downward-closed component set");
    v->d = h->d;
    v->m = h->m;
    v->device = h->device;
    v->tables = &h->dt;
    v->lo = h->dlo;
    v->span = h->dspan;
    v->stats = h->stats;
    const EvalConfig want = h->cfg[precision][form];
    if (eval_kernel_eligible(h->dt, want.kernel, precision, form)) {
        v->cfg = want;
    } else {
        // tables of the nodal kernel not built yet (this view allocates nothing):
        // the default schedule for this call, the choice kept; any other
        // ineligible choice is dropped, as hdmr_eval does
        if (!(kernel_is_nodal(want.kernel) && !h->dt.nod[form].tried)) h->cfg[precision][form] = EvalConfig();
        v->cfg = EvalConfig();
    }
    v->withhold_from = h->fi_withhold;
    return DDSG_OK;
}

HandleProfScope::HandleProfScope(hdmr_t *h_, int kind_, cudaStream_t st_) : h(h_), kind(kind_), st(st_) {
    if (!h->prof || h->capturing) return;
    a = ProfScope::take(h);
    b = ProfScope::take(h);
    if (a) cudaEventRecord(a, st);
}

HandleProfScope::~HandleProfScope() {
    if (!h->prof || !a || !b) return;
    cudaEventRecord(b, st);
    h->recs.push_back({kind, a, b});
}

int set_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace ddsg

