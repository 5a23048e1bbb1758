// ddsg_nodal.cu -- the staged nodal-slab evaluation of the DDSG interpolant
// (kernel 5): planning of its tables, their node values, and the kernel.
//
// The interpolant of a two-dimensional component u = {i, j} (Sec. 3.1, eq. 3.6)
// is s_u(x) = sum_p alpha_p phi_p(x_i) phi_p(x_j) over its points p. Grouping
// the points by their level b and cell cb in one dimension (the slab dimension,
// here called s) leaves, for a query in that cell,
//     s_u(x) = sum_b phi_{b,cb(x_s)}(x_s) * H_{b,cb(x_s)}(x_n),
// where H_{b,cb}(y) = sum of alpha_p phi_p(y) over the group's points is a 1D
// piecewise-linear function of the other (nodal) coordinate with kinks only on
// the nodes of its finest level A. H is therefore stored exactly by its values
// at the 2^(A-1) + 1 nodes k / 2^(A-1), and a query reads the two node values
// around x_n and interpolates linearly. For the d = 100 grids this is ~9.5 node
// rows per query and component instead of 16 level-tuple rows. The result is
// the same function (eq. 4.2 / the slice-free form) evaluated in another basis;
// only the rounding differs.
//
// Shared memory: the FP32 node rows of a component are staged by a bulk copy
// like the surplus rows of kernels 2-4. Rows are padded to a multiple of 32
// floats (128 bytes) and each lane reads the 16-byte chunks of its rows in an
// order rotated by its lane index within the quarter-warp, so the 8 lanes of a
// quarter-warp always read 8 different bank groups: a warp-wide 16-byte load
// costs 4 wavefronts whatever rows the 32 queries select (no bank conflicts).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <map>
#include <vector>

#include "ddsg_alloc.h"
#include "ddsg_eval.cuh"
#include "ddsg_internal.h"
#include "ddsg_tma.cuh"

namespace ddsg {

namespace {

constexpr int kNodDirMax = 1024;        // directory entries of one component
constexpr int kNodRowsMax = 1 << 20;    // node rows of one component
constexpr int kNodLevelMax = 20;        // finest nodal level A
constexpr uint32_t kNone = 0xffffu;     // "no dimension" in the dims record

uint32_t ncell(int l) { return l <= 1 ? 1u : (l == 2 ? 2u : (1u << (l - 2))); }
uint32_t cell_of(int l, uint32_t i) { return l <= 1 ? 0u : (l == 2 ? i / 2u : (i - 1u) / 2u); }

// One component's plan for a given slab dimension (index into its dims, or -1).
struct Plan {
    bool ok = false;
    double erows = 0;                        // expected node rows read per query
    int64_t rows = 0;
    std::vector<int> slab_levels;            // ascending
    // per (b, cb) with points: level A and the member points (local ids)
    std::map<std::pair<int, uint32_t>, std::pair<int, std::vector<int64_t>>> groups;
    int ndir = 0;
};

Plan plan_component(const NodalComp &c, const std::vector<int64_t> &sel, int sdim) {
    Plan P;
    const int k = c.k;
    const int ndim = k == 2 ? 1 - sdim : (k == 1 ? 0 : -1);
    for (int64_t p : sel) {
        int b = 0;
        uint32_t cb = 0;
        if (sdim >= 0) {
            b = c.lv[p * k + sdim];
            cb = cell_of(b, c.ix[p * k + sdim]);
        }
        const int a = ndim >= 0 ? c.lv[p * k + ndim] : 1;
        auto &g = P.groups[{b, cb}];
        g.first = std::max(g.first, a);
        g.second.push_back(p);
    }
    int64_t rows = 0;
    double er = 0;
    std::vector<int> lev;
    for (auto &kv : P.groups) {
        const int A = kv.second.first;
        if (A > kNodLevelMax) return P;
        rows += (1ll << (A - 1)) + 1;
        er += 2.0 / ncell(kv.first.first);
        if (lev.empty() || lev.back() != kv.first.first) lev.push_back(kv.first.first);
    }
    int ndir = 0;
    for (int b : lev) ndir += (int)ncell(b);
    if (ndir > kNodDirMax || rows > kNodRowsMax) return P;
    P.ok = true;
    P.erows = er;
    P.rows = rows;
    P.slab_levels = lev;
    P.ndir = ndir;
    return P;
}

template <typename T>
int upload(T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return DDSG_OK;
    if (dev_alloc(dst, sizeof(T) * src.size()) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DDSG_ERR_OOM, "nodal tables: device memory unavailable");
    }
    if (cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DDSG_ERR_CUDA, "nodal tables: copy to the device failed");
    }
    return DDSG_OK;
}

}  // namespace

void nodal_free(DevNodal &nd) {
    cudaFree(nd.rec);
    cudaFree(nd.rec2);
    cudaFree(nd.meta);
    cudaFree(nd.v64);
    cudaFree(nd.v32);
    cudaFree(nd.nrow);
    cudaFree(nd.grp);
    cudaFree(nd.gpts);
    nd = DevNodal();
}

int nodal_build(int m, int form, const std::vector<NodalComp> &comps, const std::vector<int32_t> &dpos,
                DevNodal &out) {
    nodal_free(out);
    out.tried = 1;
    const bool paper = form == DDSG_FORM_PAPER;
    const int mp64 = (m + 1) & ~1;
    const int rs32 = m > 16 ? (m + 31) & ~31 : (m + 3) & ~3;
    std::vector<int4> rec, rec2, nrow, gpts;
    std::vector<int2> meta, grp;
    int64_t rows_total = 0;
    int64_t meta_max = 0, rows_max = 0;
    for (int ci = 0; ci < (int)comps.size(); ++ci) {
        const NodalComp &c = comps[ci];
        if (c.k > 2) return DDSG_OK;                       // not eligible: out.ok stays 0
        if (paper && c.b == 0.0) continue;
        if (c.b != (double)(int)c.b) return DDSG_OK;
        std::vector<int64_t> sel;
        for (int64_t p = 0; p < c.npts; ++p) {
            bool in = true;
            if (!paper)
                for (int j = 0; j < c.k; ++j) in = in && c.lv[p * c.k + j] >= 2;
            if (in) sel.push_back(p);
        }
        if (sel.empty()) continue;                         // contributes nothing in this form
        Plan P;
        int sdim = -1;
        if (c.k == 2) {
            Plan p0 = plan_component(c, sel, 0), p1 = plan_component(c, sel, 1);
            const bool use1 = p1.ok && (!p0.ok || p1.erows < p0.erows ||
                                        (p1.erows == p0.erows && p1.rows < p0.rows));
            P = use1 ? std::move(p1) : std::move(p0);
            sdim = use1 ? 1 : 0;
        } else {
            P = plan_component(c, sel, -1);
        }
        if (!P.ok) return DDSG_OK;
        const int ndim = c.k == 2 ? 1 - sdim : (c.k == 1 ? 0 : -1);
        // meta block: slab entries, then the directory of each slab level
        const int64_t mb = (int64_t)meta.size();
        const int nslab = (int)P.slab_levels.size();
        std::vector<int2> blk(nslab + P.ndir, make_int2(-1, 0));
        int dir = nslab;
        std::map<int, int> dir_of;
        for (int s = 0; s < nslab; ++s) {
            const int b = P.slab_levels[s];
            blk[s] = make_int2(b, dir);
            dir_of[b] = dir;
            dir += (int)ncell(b);
        }
        int64_t row = 0;
        for (auto &kv : P.groups) {
            const int b = kv.first.first;
            const uint32_t cb = kv.first.second;
            const int A = kv.second.first;
            blk[dir_of[b] + cb] = make_int2((int)row, A);
            const int64_t g = (int64_t)grp.size();
            const int64_t gb = (int64_t)gpts.size();
            for (int64_t p : kv.second.second) {
                const int l = ndim >= 0 ? c.lv[p * c.k + ndim] : 1;
                const uint32_t i = ndim >= 0 ? c.ix[p * c.k + ndim] : 1u;
                gpts.push_back(make_int4(dpos[c.first + p], l, (int)i, 0));
            }
            grp.push_back(make_int2((int)gb, (int)gpts.size()));
            const int64_t nn = (1ll << (A - 1)) + 1;
            for (int64_t kk = 0; kk < nn; ++kk) nrow.push_back(make_int4((int)g, (int)kk, A, 0));
            row += nn;
        }
        if ((int64_t)gpts.size() >= INT_MAX || rows_total + row >= INT_MAX) return DDSG_OK;
        if (blk.size() & 1) blk.push_back(make_int2(0, 0));  // 16-byte blocks
        meta.insert(meta.end(), blk.begin(), blk.end());
        const int nmeta = nslab + P.ndir;
        rec.push_back(make_int4((int)mb, nmeta | (nslab << 16), (int)rows_total, (int)row));
        const uint32_t dn = ndim >= 0 ? (uint32_t)c.dims[ndim] : kNone;
        const uint32_t ds = sdim >= 0 ? (uint32_t)c.dims[sdim] : kNone;
        rec2.push_back(make_int4(ci, (int)(dn | (ds << 16)), (int)c.b, 0));
        out.erows += P.erows;
        meta_max = std::max<int64_t>(meta_max, ((int64_t)nmeta * 8 + 15) & ~15ll);
        rows_max = std::max<int64_t>(rows_max, row);
        rows_total += row;
        if (meta.size() >= (size_t)INT_MAX) return DDSG_OK;
    }
    const double erows = out.erows;
    out.n = (int32_t)rec.size();
    out.rows = rows_total;
    out.erows = erows;
    out.rs32 = rs32;
    out.meta_bytes = (int32_t)((meta_max + 127) & ~127ll);
    out.stage_bytes[DDSG_F64] = out.meta_bytes + rows_max * mp64 * 8;
    out.stage_bytes[DDSG_F32C] = out.meta_bytes + rows_max * rs32 * 4;
    out.ngrp = (int64_t)grp.size();
    out.ngpts = (int64_t)gpts.size();
    int rc;
    if ((rc = upload(&out.rec, rec)) || (rc = upload(&out.rec2, rec2)) || (rc = upload(&out.meta, meta)) ||
        (rc = upload(&out.nrow, nrow)) || (rc = upload(&out.grp, grp)) || (rc = upload(&out.gpts, gpts))) {
        nodal_free(out);
        out.tried = 1;
        return rc;
    }
    if (rows_total > 0) {
        if (dev_alloc(&out.v64, sizeof(double) * (size_t)rows_total * mp64) != cudaSuccess ||
            dev_alloc(&out.v32, sizeof(float) * (size_t)rows_total * rs32) != cudaSuccess) {
            cudaGetLastError();
            nodal_free(out);
            out.tried = 1;
            return set_error(DDSG_ERR_OOM, "nodal tables: device memory for the node values unavailable");
        }
        // padding columns stay zero
        if (cudaMemset(out.v64, 0, sizeof(double) * (size_t)rows_total * mp64) != cudaSuccess ||
            cudaMemset(out.v32, 0, sizeof(float) * (size_t)rows_total * rs32) != cudaSuccess) {
            cudaGetLastError();
            nodal_free(out);
            out.tried = 1;
            return set_error(DDSG_ERR_CUDA, "nodal tables: clearing the node values failed");
        }
    }
    out.ok = 1;
    return DDSG_OK;
}

// ---------------------------------------------------------------------------
// node values (FP64 from the FP64 surpluses, then the FP32 copy)
// ---------------------------------------------------------------------------

// Hat of point (l, i) at the dyadic node y (exact in FP64 for l, A <= 20):
// level 1 the constant 1, level 2 the boundary hats of nodes 0 and 1, level
// l >= 3 the interior hat of node i / 2^(l-1) (Sec. 3.1 with boundary levels).
__device__ __forceinline__ double node_hat(int l, int i, double y) {
    if (l <= 1) return 1.0;
    if (l == 2) return i == 0 ? fmax(0.0, 1.0 - 2.0 * y) : fmax(0.0, 2.0 * y - 1.0);
    return fmax(0.0, 1.0 - fabs(ldexp(y, l - 1) - (double)i));
}

// v64[r][o] = sum over the points of row r's cell group of alpha_p[o] * hat_p(node),
// one thread per (node row, output), points in group order.
__global__ void nodalize_kernel(const int4 *__restrict__ nrow, int64_t R, const int2 *__restrict__ grp,
                                const int4 *__restrict__ gpts, const double *__restrict__ alpha64, int mp64,
                                int m, double *__restrict__ v64) {
    const int64_t total = R * (int64_t)m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / m;
        const int o = (int)(e - r * m);
        const int4 nr = nrow[r];
        const double y = ldexp((double)nr.y, -(nr.z - 1));
        const int2 g = grp[nr.x];
        double acc = 0.0;
        for (int q = g.x; q < g.y; ++q) {
            const int4 gp = gpts[q];
            const double h = node_hat(gp.y, gp.z, y);
            if (h != 0.0) acc = fma(h, alpha64[(int64_t)gp.x * mp64 + o], acc);
        }
        v64[r * mp64 + o] = acc;
    }
}

__global__ void nodal_to_f32_kernel(const double *__restrict__ v64, int mp64, float *__restrict__ v32, int rs32,
                                    int64_t R, int m) {
    const int64_t total = R * (int64_t)m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / m;
        const int o = (int)(e - r * m);
        v32[r * rs32 + o] = __double2float_rn(v64[r * mp64 + o]);
    }
}

cudaError_t launch_nodalize(const DevNodal &nd, const double *alpha64, int mp64, int m, cudaStream_t st) {
    if (!nd.ok || nd.rows <= 0) return cudaSuccess;
    const int64_t total = nd.rows * (int64_t)m;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    nodalize_kernel<<<(unsigned)blocks, 256, 0, st>>>(nd.nrow, nd.rows, nd.grp, nd.gpts, alpha64, mp64, m, nd.v64);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nodal_to_f32_kernel<<<(unsigned)blocks, 256, 0, st>>>(nd.v64, mp64, nd.v32, nd.rs32, nd.rows, m);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// the staged nodal-slab evaluation kernel
// ---------------------------------------------------------------------------

// Block shape: GR output windows per block over the same QB queries (one warp
// group per window); a thread owns one query and MC outputs of it.
template <int GR>
struct NodShape {
    static constexpr int QB = GR == 1 ? 256 : 192;
    static constexpr int NT = QB * GR;
    static constexpr int QW = QB / 32;
};

template <int PREC>
__device__ __forceinline__ typename Types<PREC>::W scaled(uint64_t N, int e) {
    if constexpr (PREC == DDSG_F64) return basis_to_f64(N, e);
    else return basis_to_f32(N, e);
}

// Cell cb of slab level b containing the fixed-point coordinate X and the hat
// value there (zero on a cell face, where the hat vanishes). b = 0 stands for a
// component without a slab dimension (a single cell, value 1).
template <int PREC>
__device__ __forceinline__ void slab_basis(uint64_t X, int b, uint32_t &cb, typename Types<PREC>::W &phi) {
    using W = typename Types<PREC>::W;
    if (b <= 1) {
        cb = 0;
        phi = (W)1;
        return;
    }
    if (b == 2) {
        const uint64_t half = 1ull << 61;
        cb = X >= half ? 1u : 0u;
        phi = scaled<PREC>(X >= half ? X - half : half - X, 61);
        return;
    }
    const int sh = 64 - b;
    uint64_t cell = X >> sh;
    const uint64_t nmax = (1ull << (b - 2)) - 1;
    cell = cell > nmax ? nmax : cell;
    const uint64_t F = X - (cell << sh);
    const uint64_t R = (1ull << sh) - F;
    cb = (uint32_t)cell;
    phi = scaled<PREC>(F < R ? F : R, sh - 1);
}

// Interval kk of the level-A node grid (nodes k / 2^(A-1)) holding X and the
// position t in [0, 1] inside it (the last interval holds X = 1).
template <int PREC>
__device__ __forceinline__ void node_pos(uint64_t X, int A, uint32_t &kk, typename Types<PREC>::W &t) {
    const int sh = 63 - A;
    uint64_t k = X >> sh;
    const uint64_t kmax = (1ull << (A - 1)) - 1;
    k = k > kmax ? kmax : k;
    kk = (uint32_t)k;
    t = scaled<PREC>(X - (k << sh), sh);
}

// One staging buffer per processed component j (buffer j % nbuf):
//   [0, meta_bytes)            its meta block (slab entries and directory),
//   [meta_bytes, ...)          its node rows (stride rs elements).
// The pipeline (full / empty mbarriers, thread 0 staging component i + 2 once
// every warp is done with i + 2 - nbuf, bounded waits, the withheld-copy test
// switch) is that of eval_tma_kernel. No shared memory is written by the
// threads, so warps need no barrier among themselves. MC = 32 with FP32 is the
// rotated layout: a thread's 32 outputs are 8 16-byte chunks of a 128-byte
// aligned window of the row, read in the order (s + lane) mod 8, and its
// accumulator slot s holds chunk (s + lane) mod 8.
template <int PREC, int MC, int GR>
__global__ void __launch_bounds__(NodShape<GR>::NT, 1) eval_nodal_kernel(const EvalParams p, int buf_bytes, int nbuf) {
    using T = Types<PREC>;
    using W = typename T::W;
    using V = typename T::V;
    constexpr bool ROT = PREC == DDSG_F32C && MC == 32;
    constexpr int VW = T::VW;
    constexpr int G = MC / VW;
    constexpr int QB = NodShape<GR>::QB;
    constexpr int QW = NodShape<GR>::QW;
    constexpr int kWarps = NodShape<GR>::NT / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + TMA_NBUF_MAX;
    unsigned char *bufbase = smem + 128;

    const DevNodal &N = p.t.nod[p.form];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int grp = warp / QW;
    const int qw = warp - grp * QW;
    const int qi = qw * 32 + lane;
    const int64_t q = (int64_t)blockIdx.x * QB + qi;
    const int64_t qc = q < p.n ? q : p.n - 1;
    const bool valid = q < p.n;
    const bool bad = !valid || p.flags[q] != 0;
    const bool paper = p.form == DDSG_FORM_PAPER;
    const int m = p.m;
    const int rs = PREC == DDSG_F64 ? p.t.mp64 : N.rs32;
    const int m0 = (blockIdx.y * GR + grp) * MC;
    const bool wact = m0 < rs;                 // this window holds outputs
    const int nproc = N.n;
    const int meta_bytes = N.meta_bytes;
    const W *gvals;
    if constexpr (PREC == DDSG_F64) gvals = N.v64;
    else gvals = N.v32;

    auto issue = [&](int j, int4 rec) {
        if (j >= p.issue_end) return;
        const int b = j % nbuf;
        const uint32_t nmeta = (uint32_t)rec.y & 0xffffu;
        const uint32_t mbytes = (nmeta * 8u + 15u) & ~15u;
        const uint32_t rbytes = (uint32_t)rec.w * (uint32_t)rs * (uint32_t)sizeof(W);
        if (!DDSG_CK(mbytes <= (uint32_t)meta_bytes && (int64_t)meta_bytes + rbytes <= (int64_t)buf_bytes &&
                         rec.z >= 0 && (int64_t)rec.z + rec.w <= N.rows,
                     CK_STAGE))
            return;
        unsigned char *dst = bufbase + (size_t)b * buf_bytes;
        mbar_expect_tx(&full[b], mbytes + rbytes);
        tma_bulk_g2s(dst, N.meta + rec.x, mbytes, &full[b]);
        if (rbytes) tma_bulk_g2s(dst + meta_bytes, gvals + (int64_t)rec.z * rs, rbytes, &full[b]);
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
        if (nproc > 0) issue(0, N.rec[0]);
        if (nproc > 1) issue(1, N.rec[1]);
        nissued = nproc < 2 ? nproc : 2;
        if (nproc > 2) rec_next = N.rec[2];
    }

    Result<PREC, MC> r;
    r.init();
    bool failed = false;
    int pfail = 0;
    // coordinates of the current component's nodal and slab dimensions, and the
    // records of the current and the next component
    auto coord = [&](uint32_t dim) -> uint64_t {
        if (dim == kNone) return 0ull;
        return DDSG_CK(dim < (uint32_t)p.d, CK_DIM) ? p.X[(int64_t)dim * p.n + qc] : 0ull;
    };
    int4 rc = nproc > 0 ? N.rec[0] : make_int4(0, 0, 0, 0);
    int4 r2c = nproc > 0 ? N.rec2[0] : make_int4(0, 0, 0, 0);
    int4 r2n = nproc > 1 ? N.rec2[1] : make_int4(0, 0, 0, 0);
    uint64_t Xn = coord((uint32_t)r2c.y & 0xffffu), Xs = coord((uint32_t)r2c.y >> 16);
    const int l8 = lane & 7;
    int b = 0;
    uint32_t ph = 0;
    for (int i = 0; i < nproc; ++i) {
        int4 rcn = make_int4(0, 0, 0, 0), r2nn = make_int4(0, 0, 0, 0);
        uint64_t Xnn = 0, Xsn = 0;
        if (i + 1 < nproc) {
            rcn = N.rec[i + 1];
            Xnn = coord((uint32_t)r2n.y & 0xffffu);
            Xsn = coord((uint32_t)r2n.y >> 16);
        }
        if (i + 2 < nproc) r2nn = N.rec2[i + 2];
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[b], ph));
        if (!ok || pfail) {
            failed = true;
            if (lane == 0 && p.err) atomicAdd(p.err, 1ull);
            break;
        }
        const unsigned char *buf = bufbase + (size_t)b * buf_bytes;
        const int2 *meta = reinterpret_cast<const int2 *>(buf);
        const W *srow = reinterpret_cast<const W *>(buf + meta_bytes);
        const int nslab = rc.y >> 16;
        const int nmeta = rc.y & 0xffff;   // bounds of the checked build's tests
        const int nrows = rc.w;
        (void)nmeta;
        (void)nrows;
        const W wb = paper ? (W)r2c.z : (W)1;
        // warp-uniform: every lane runs the slab loop (it votes); a lane with no
        // valid query or a non-finite one is inactive, with weights zero
        if (wact) {
            for (int sl = 0; sl < nslab; ++sl) {
                const int2 se = meta[sl];
                uint32_t cb;
                W phi;
                slab_basis<PREC>(Xs, se.x, cb, phi);
                const int di = se.y + (int)cb;
                const int2 de = DDSG_CK(di >= 0 && di < nmeta, CK_STAGE) ? meta[di] : make_int2(-1, 1);
                bool act = !bad && de.x >= 0 && phi != (W)0;
                if (!__any_sync(0xffffffffu, act)) continue;
                uint32_t kk = 0;
                W t = (W)0;
                node_pos<PREC>(Xn, act ? de.y : 1, kk, t);
                int32_t r0 = act ? de.x + (int32_t)kk : 0;
                if (!DDSG_CK(r0 >= 0 && r0 + 1 < nrows, CK_ROW)) {
                    act = false;
                    r0 = 0;
                }
                const W pw = phi * wb;
                const W w1 = act ? pw * t : (W)0;
                const W w0 = act ? pw * ((W)1 - t) : (W)0;
                const V *R0 = reinterpret_cast<const V *>(srow + (int64_t)r0 * rs + m0);
                const V *R1 = reinterpret_cast<const V *>(srow + (int64_t)(r0 + 1) * rs + m0);
                auto &acc = r.partial();
                if constexpr (ROT) {
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        const int c = (s + l8) & 7;
                        const V a0 = R0[c], a1 = R1[c];
                        acc[4 * s + 0] = fmaf(w1, a1.x, fmaf(w0, a0.x, acc[4 * s + 0]));
                        acc[4 * s + 1] = fmaf(w1, a1.y, fmaf(w0, a0.y, acc[4 * s + 1]));
                        acc[4 * s + 2] = fmaf(w1, a1.z, fmaf(w0, a0.z, acc[4 * s + 2]));
                        acc[4 * s + 3] = fmaf(w1, a1.w, fmaf(w0, a0.w, acc[4 * s + 3]));
                    }
                } else {
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (m0 + g * VW < rs) {
                            const V a0 = R0[g], a1 = R1[g];
                            if constexpr (VW == 4) {
                                acc[4 * g + 0] = fmaf(w1, a1.x, fmaf(w0, a0.x, acc[4 * g + 0]));
                                acc[4 * g + 1] = fmaf(w1, a1.y, fmaf(w0, a0.y, acc[4 * g + 1]));
                                acc[4 * g + 2] = fmaf(w1, a1.z, fmaf(w0, a0.z, acc[4 * g + 2]));
                                acc[4 * g + 3] = fmaf(w1, a1.w, fmaf(w0, a0.w, acc[4 * g + 3]));
                            } else {
                                acc[2 * g + 0] = fma(w1, a1.x, fma(w0, a0.x, acc[2 * g + 0]));
                                acc[2 * g + 1] = fma(w1, a1.y, fma(w0, a0.y, acc[2 * g + 1]));
                            }
                        }
                    }
                }
            }
            r.fold();
        }
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
                if (j + 1 < nproc) rec_next = N.rec[j + 1];
            }
        }
        pfail = __shfl_sync(0xffffffffu, pf, 0);
        rc = rcn;
        r2c = r2n;
        r2n = r2nn;
        Xn = Xnn;
        Xs = Xsn;
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
    if (!valid || !wact) return;
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int o = 0; o < MC; ++o) {
        const int oo = ROT ? m0 + (((o >> 2) + l8) & 7) * 4 + (o & 3) : m0 + o;
        if (oo < m) p.y[q * m + oo] = (bad || failed) ? nanv : r.value(o);
    }
}

// ---------------------------------------------------------------------------
// FP32-compensated nodal-slab kernel with paired FP32 arithmetic: the node rows
// of a thread's 32-output window are read as eight 16-byte chunks in the order
// s ^ (lane mod 8) (s = 0..7), so the 8 lanes of a quarter-warp read 8 different
// bank groups; each chunk feeds two fma.rn.f32x2 per row. The per-component
// partials (pairs of FP32) are folded every second component into a Kahan
// total (add / sub .rn.f32x2, no contraction).
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Slab cell and hat value from x31 = X >> 31 (31 fraction bits) for slab levels
// b <= 10 (at least 23 bits of the position inside the cell), else from X.
__device__ __forceinline__ void slab_basis_f32(uint64_t X, uint32_t x31, int b, uint32_t &cb, float &phi) {
    if (b <= 1) {
        cb = 0;
        phi = 1.0f;
    } else if (b == 2) {
        const uint32_t half = 1u << 30;
        cb = x31 >= half ? 1u : 0u;
        phi = __uint2float_rn(x31 >= half ? x31 - half : half - x31) * pow2m_f(30);
    } else if (b <= 10) {
        const int sh = 33 - b;
        uint32_t cell = x31 >> sh;
        const uint32_t nmax = (1u << (b - 2)) - 1u;
        cell = cell > nmax ? nmax : cell;
        const uint32_t F = x31 - (cell << sh);
        const uint32_t R = (1u << sh) - F;
        cb = cell;
        phi = __uint2float_rn(F < R ? F : R) * pow2m_f(sh - 1);
    } else {
        slab_basis<DDSG_F32C>(X, b, cb, phi);
    }
}

// Node interval and position from x31 for nodal levels A <= 10, else from X.
__device__ __forceinline__ void node_pos_f32(uint64_t X, uint32_t x31, int A, uint32_t &kk, float &t) {
    if (A <= 10) {
        const int sh = 32 - A;
        uint32_t k = x31 >> sh;
        const uint32_t kmax = (1u << (A - 1)) - 1u;
        k = k > kmax ? kmax : k;
        kk = k;
        t = __uint2float_rn(x31 - (k << sh)) * pow2m_f(sh);
    } else {
        node_pos<DDSG_F32C>(X, A, kk, t);
    }
}

struct NodProbe {
    int32_t r0;     // first of the two node rows (staged row index), 0 when inactive
    float w0, w1;   // weights of rows r0 and r0 + 1 (zero when inactive)
    bool act;
};

// Slab sl of the staged component: cell, directory entry, node interval, weights.
__device__ __forceinline__ NodProbe nodal_probe(const int2 *meta, int sl, int nmeta, int nrows, uint64_t Xs,
                                                uint32_t xs31, uint64_t Xn, uint32_t xn31, bool bad, float wb) {
    NodProbe pr;
    const int2 se = meta[sl];
    uint32_t cb;
    float phi;
    slab_basis_f32(Xs, xs31, se.x, cb, phi);
    const int di = se.y + (int)cb;
    const int2 de = DDSG_CK(di >= 0 && di < nmeta, CK_STAGE) ? meta[di] : make_int2(-1, 1);
    pr.act = !bad && de.x >= 0 && phi != 0.0f;
    uint32_t kk = 0;
    float t = 0.0f;
    node_pos_f32(Xn, xn31, pr.act ? de.y : 1, kk, t);
    pr.r0 = pr.act ? de.x + (int32_t)kk : 0;
    if (!DDSG_CK(pr.r0 >= 0 && pr.r0 + 1 < nrows, CK_ROW)) {
        pr.act = false;
        pr.r0 = 0;
    }
    (void)nmeta;
    (void)nrows;
    const float pw = phi * wb;
    pr.w1 = pr.act ? pw * t : 0.0f;
    pr.w0 = pr.act ? pw * (1.0f - t) : 0.0f;
    return pr;
}

template <int GR>
__global__ void __launch_bounds__(NodShape<GR>::NT, 1) eval_nodal_f32x2_kernel(const EvalParams p, int buf_bytes,
                                                                              int nbuf) {
    constexpr int QB = NodShape<GR>::QB;
    constexpr int QW = NodShape<GR>::QW;
    constexpr int kWarps = NodShape<GR>::NT / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + TMA_NBUF_MAX;
    unsigned char *bufbase = smem + 128;

    const DevNodal &N = p.t.nod[p.form];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int grp = warp / QW;
    const int qw = warp - grp * QW;
    const int qi = qw * 32 + lane;
    const int64_t q = (int64_t)blockIdx.x * QB + qi;
    const int64_t qc = q < p.n ? q : p.n - 1;
    const bool valid = q < p.n;
    const bool bad = !valid || p.flags[q] != 0;
    const bool paper = p.form == DDSG_FORM_PAPER;
    const int m = p.m;
    const int rs = N.rs32;
    const int m0 = (blockIdx.y * GR + grp) * 32;
    const bool wact = m0 < rs;
    const int nproc = N.n;
    const int meta_bytes = N.meta_bytes;
    const int l8 = lane & 7;

    auto issue = [&](int j, int4 rec) {
        if (j >= p.issue_end) return;
        const int b = j % nbuf;
        const uint32_t nmeta = (uint32_t)rec.y & 0xffffu;
        const uint32_t mbytes = (nmeta * 8u + 15u) & ~15u;
        const uint32_t rbytes = (uint32_t)rec.w * (uint32_t)rs * 4u;
        if (!DDSG_CK(mbytes <= (uint32_t)meta_bytes && (int64_t)meta_bytes + rbytes <= (int64_t)buf_bytes &&
                         rec.z >= 0 && (int64_t)rec.z + rec.w <= N.rows,
                     CK_STAGE))
            return;
        unsigned char *dst = bufbase + (size_t)b * buf_bytes;
        mbar_expect_tx(&full[b], mbytes + rbytes);
        tma_bulk_g2s(dst, N.meta + rec.x, mbytes, &full[b]);
        if (rbytes) tma_bulk_g2s(dst + meta_bytes, N.v32 + (int64_t)rec.z * rs, rbytes, &full[b]);
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
        if (nproc > 0) issue(0, N.rec[0]);
        if (nproc > 1) issue(1, N.rec[1]);
        nissued = nproc < 2 ? nproc : 2;
        if (nproc > 2) rec_next = N.rec[2];
    }

    uint64_t acc[16], ks[16], kc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = ks[u] = kc[u] = 0ull;
    auto fold = [&]() {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint64_t yk = f2_sub(acc[u], kc[u]);
            const uint64_t tk = f2_add(ks[u], yk);
            kc[u] = f2_sub(f2_sub(tk, ks[u]), yk);
            ks[u] = tk;
            acc[u] = 0ull;
        }
    };
    bool failed = false;
    int pfail = 0;
    auto coord = [&](uint32_t dim) -> uint64_t {
        if (dim == kNone) return 0ull;
        return DDSG_CK(dim < (uint32_t)p.d, CK_DIM) ? p.X[(int64_t)dim * p.n + qc] : 0ull;
    };
    int4 rc = nproc > 0 ? N.rec[0] : make_int4(0, 0, 0, 0);
    int4 r2c = nproc > 0 ? N.rec2[0] : make_int4(0, 0, 0, 0);
    int4 r2n = nproc > 1 ? N.rec2[1] : make_int4(0, 0, 0, 0);
    uint64_t Xn = coord((uint32_t)r2c.y & 0xffffu), Xs = coord((uint32_t)r2c.y >> 16);
    int b = 0;
    uint32_t ph = 0;
    for (int i = 0; i < nproc; ++i) {
        int4 rcn = make_int4(0, 0, 0, 0), r2nn = make_int4(0, 0, 0, 0);
        uint64_t Xnn = 0, Xsn = 0;
        if (i + 1 < nproc) {
            rcn = N.rec[i + 1];
            Xnn = coord((uint32_t)r2n.y & 0xffffu);
            Xsn = coord((uint32_t)r2n.y >> 16);
        }
        if (i + 2 < nproc) r2nn = N.rec2[i + 2];
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[b], ph));
        if (!ok || pfail) {
            failed = true;
            if (lane == 0 && p.err) atomicAdd(p.err, 1ull);
            break;
        }
        const unsigned char *buf = bufbase + (size_t)b * buf_bytes;
        const int2 *meta = reinterpret_cast<const int2 *>(buf);
        const unsigned char *srow = buf + meta_bytes + (size_t)m0 * 4;   // this window of row 0
        const int nslab = rc.y >> 16;
        const int nmeta = rc.y & 0xffff;
        const int nrows = rc.w;
        const float wb = paper ? (float)r2c.z : 1.0f;
        const uint32_t xs31 = (uint32_t)(Xs >> 31), xn31 = (uint32_t)(Xn >> 31);
        const int rstride = rs * 4;
        // warp-uniform: every lane runs the slab loop (it votes); lanes without a
        // valid, finite query are inactive (weights zero, row 0)
        if (wact && nslab > 0) {
            NodProbe pr = nodal_probe(meta, 0, nmeta, nrows, Xs, xs31, Xn, xn31, bad, wb);
            for (int sl = 0; sl < nslab; ++sl) {
                NodProbe nx;
                if (sl + 1 < nslab) nx = nodal_probe(meta, sl + 1, nmeta, nrows, Xs, xs31, Xn, xn31, bad, wb);
                if (__any_sync(0xffffffffu, pr.act)) {
                    const unsigned char *R0 = srow + (size_t)pr.r0 * rstride;
                    const uint64_t w0 = f2_pack(pr.w0, pr.w0), w1 = f2_pack(pr.w1, pr.w1);
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        const int off = (s ^ l8) << 4;
                        const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(R0 + off);
                        const ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(R0 + rstride + off);
                        acc[2 * s] = f2_fma(w1, a1.x, f2_fma(w0, a0.x, acc[2 * s]));
                        acc[2 * s + 1] = f2_fma(w1, a1.y, f2_fma(w0, a0.y, acc[2 * s + 1]));
                    }
                }
                pr = nx;
            }
        }
        if ((i & 1) || i + 1 == nproc) fold();
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
                if (j + 1 < nproc) rec_next = N.rec[j + 1];
            }
        }
        pfail = __shfl_sync(0xffffffffu, pf, 0);
        rc = rcn;
        r2c = r2n;
        r2n = r2nn;
        Xn = Xnn;
        Xs = Xsn;
        if (++b == nbuf) {
            b = 0;
            ph ^= 1u;
        }
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = nissued > nbuf ? nissued - nbuf : 0; j < nissued; ++j)
            if (j < p.issue_end) mbar_wait_bounded(&full[j % nbuf], (uint32_t)((j / nbuf) & 1));
    }
    if (!valid || !wact) return;
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int o0 = m0 + ((s ^ l8) << 2);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float s0, s1, c0, c1;
            f2_unpack(ks[2 * s + h], s0, s1);
            f2_unpack(kc[2 * s + h], c0, c1);
            const int o = o0 + 2 * h;
            if (o < m) p.y[q * m + o] = (bad || failed) ? nanv : (double)s0 - (double)c0;
            if (o + 1 < m) p.y[q * m + o + 1] = (bad || failed) ? nanv : (double)s1 - (double)c1;
        }
    }
}

// ---------------------------------------------------------------------------
// The same kernel with the Kahan totals in tensor memory (kernel 6). Between
// folds a thread keeps only its 32-output partial in registers; the totals s
// and compensations c (64 FP32 per thread) live in tensor memory, which this
// path otherwise leaves unused. Each warp owns 64 columns of its lane quarter
// (lanes 32 (w mod 4) ..): 16 warps x 64 columns = 256 columns per block. A
// fold reads 8 outputs' (s, c) at a time (tcgen05.ld 32x32b.x8), updates them
// and writes them back (tcgen05.st), so it holds 16 more registers, not 64.
// Fewer registers allow 256 queries per block in 16 warps per SM.
// ---------------------------------------------------------------------------

constexpr int kTmQB = 256;                 // queries per block
constexpr int kTmNT = 2 * kTmQB;           // two output windows
constexpr uint32_t kTmCols = 256;          // tensor-memory columns per block

__device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tm_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint64_t u2pack(uint32_t a, uint32_t b) { return (uint64_t)a | ((uint64_t)b << 32); }

__global__ void __launch_bounds__(kTmNT, 1) eval_nodal_tmem_kernel(const EvalParams p, int buf_bytes, int nbuf) {
    constexpr int QW = kTmQB / 32;
    constexpr int kWarps = kTmNT / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + TMA_NBUF_MAX;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 96);
    unsigned char *bufbase = smem + 128;

    const DevNodal &N = p.t.nod[p.form];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int grp = warp / QW;
    const int qw = warp - grp * QW;
    const int qi = qw * 32 + lane;
    // work items (query tile of kTmQB, output window of 32), window fastest; the
    // block's two warp groups take two consecutive items, so an odd number of
    // windows leaves no group idle
    const int nwin = N.rs32 >> 5;
    const int64_t ntile = (p.n + kTmQB - 1) / kTmQB;
    const int64_t item = (int64_t)blockIdx.x * 2 + grp;
    const int64_t tile = item / nwin;
    const int64_t q = tile * kTmQB + qi;
    const int64_t qc = q < p.n ? q : p.n - 1;
    const bool valid = q < p.n;
    const bool bad = !valid || p.flags[q] != 0;
    const bool paper = p.form == DDSG_FORM_PAPER;
    const int m = p.m;
    const int rs = N.rs32;
    const int m0 = (int)(item - tile * nwin) * 32;
    const bool wact = item < ntile * nwin;
    const int nproc = N.n;
    const int meta_bytes = N.meta_bytes;
    const int l8 = lane & 7;

    auto issue = [&](int j, int4 rec) {
        if (j >= p.issue_end) return;
        const int b = j % nbuf;
        const uint32_t nmeta = (uint32_t)rec.y & 0xffffu;
        const uint32_t mbytes = (nmeta * 8u + 15u) & ~15u;
        const uint32_t rbytes = (uint32_t)rec.w * (uint32_t)rs * 4u;
        if (!DDSG_CK(mbytes <= (uint32_t)meta_bytes && (int64_t)meta_bytes + rbytes <= (int64_t)buf_bytes &&
                         rec.z >= 0 && (int64_t)rec.z + rec.w <= N.rows,
                     CK_STAGE))
            return;
        unsigned char *dst = bufbase + (size_t)b * buf_bytes;
        mbar_expect_tx(&full[b], mbytes + rbytes);
        tma_bulk_g2s(dst, N.meta + rec.x, mbytes, &full[b]);
        if (rbytes) tma_bulk_g2s(dst + meta_bytes, N.v32 + (int64_t)rec.z * rs, rbytes, &full[b]);
    };

    if (tid == 0) {
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], kWarps);
        }
        mbar_fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // this warp's 64 columns of its lane quarter: s in [0, 32), c in [32, 64)
    const uint32_t tbase = *tslot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
    {
        const uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 8; ++k) tm_st8(tbase + 8 * k, z);
        tm_wait_st();
    }
    int nissued = 0;
    int4 rec_next = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        if (nproc > 0) issue(0, N.rec[0]);
        if (nproc > 1) issue(1, N.rec[1]);
        nissued = nproc < 2 ? nproc : 2;
        if (nproc > 2) rec_next = N.rec[2];
    }

    uint64_t acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = 0ull;
    // Kahan fold of the partial into the totals in tensor memory, 8 outputs at a time
    auto fold = [&]() {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t sv[8], cv[8];
            tm_ld8(tbase + 8 * k, sv);
            tm_ld8(tbase + 32 + 8 * k, cv);
            tm_wait_ld();
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t s2 = u2pack(sv[2 * u], sv[2 * u + 1]);
                const uint64_t c2 = u2pack(cv[2 * u], cv[2 * u + 1]);
                const uint64_t yk = f2_sub(acc[4 * k + u], c2);
                const uint64_t tk = f2_add(s2, yk);
                const uint64_t cn = f2_sub(f2_sub(tk, s2), yk);
                sv[2 * u] = (uint32_t)tk;
                sv[2 * u + 1] = (uint32_t)(tk >> 32);
                cv[2 * u] = (uint32_t)cn;
                cv[2 * u + 1] = (uint32_t)(cn >> 32);
                acc[4 * k + u] = 0ull;
            }
            tm_st8(tbase + 8 * k, sv);
            tm_st8(tbase + 32 + 8 * k, cv);
        }
        tm_wait_st();
    };
    bool failed = false;
    int pfail = 0;
    auto coord = [&](uint32_t dim) -> uint64_t {
        if (dim == kNone) return 0ull;
        return DDSG_CK(dim < (uint32_t)p.d, CK_DIM) ? p.X[(int64_t)dim * p.n + qc] : 0ull;
    };
    int4 rc = nproc > 0 ? N.rec[0] : make_int4(0, 0, 0, 0);
    int4 r2c = nproc > 0 ? N.rec2[0] : make_int4(0, 0, 0, 0);
    int4 r2n = nproc > 1 ? N.rec2[1] : make_int4(0, 0, 0, 0);
    uint64_t Xn = coord((uint32_t)r2c.y & 0xffffu), Xs = coord((uint32_t)r2c.y >> 16);
    int b = 0;
    uint32_t ph = 0;
    for (int i = 0; i < nproc; ++i) {
        int4 rcn = make_int4(0, 0, 0, 0), r2nn = make_int4(0, 0, 0, 0);
        uint64_t Xnn = 0, Xsn = 0;
        if (i + 1 < nproc) {
            rcn = N.rec[i + 1];
            Xnn = coord((uint32_t)r2n.y & 0xffffu);
            Xsn = coord((uint32_t)r2n.y >> 16);
        }
        if (i + 2 < nproc) r2nn = N.rec2[i + 2];
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[b], ph));
        if (!ok || pfail) {
            failed = true;
            if (lane == 0 && p.err) atomicAdd(p.err, 1ull);
            break;
        }
        const unsigned char *buf = bufbase + (size_t)b * buf_bytes;
        const int2 *meta = reinterpret_cast<const int2 *>(buf);
        const unsigned char *srow = buf + meta_bytes + (size_t)m0 * 4;
        const int nslab = rc.y >> 16;
        const int nmeta = rc.y & 0xffff;
        const int nrows = rc.w;
        const float wb = paper ? (float)r2c.z : 1.0f;
        const uint32_t xs31 = (uint32_t)(Xs >> 31), xn31 = (uint32_t)(Xn >> 31);
        const int rstride = rs * 4;
        if (wact && nslab > 0) {
            NodProbe pr = nodal_probe(meta, 0, nmeta, nrows, Xs, xs31, Xn, xn31, bad, wb);
            for (int sl = 0; sl < nslab; ++sl) {
                NodProbe nx;
                if (sl + 1 < nslab) nx = nodal_probe(meta, sl + 1, nmeta, nrows, Xs, xs31, Xn, xn31, bad, wb);
                if (__any_sync(0xffffffffu, pr.act)) {
                    const unsigned char *R0 = srow + (size_t)pr.r0 * rstride;
                    const uint64_t w0 = f2_pack(pr.w0, pr.w0), w1 = f2_pack(pr.w1, pr.w1);
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        const int off = (s ^ l8) << 4;
                        const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(R0 + off);
                        const ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(R0 + rstride + off);
                        acc[2 * s] = f2_fma(w1, a1.x, f2_fma(w0, a0.x, acc[2 * s]));
                        acc[2 * s + 1] = f2_fma(w1, a1.y, f2_fma(w0, a0.y, acc[2 * s + 1]));
                    }
                }
                pr = nx;
            }
        }
        if ((i & 1) || i + 1 == nproc) fold();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
        int pf = 0;
        if (tid == 0 && i + 2 < nproc) {
            const int j = i + 2;
            if (j >= nbuf && !mbar_wait_bounded(&empty[j % nbuf], (uint32_t)(((j - nbuf) / nbuf) & 1))) {
                pf = 1;
            } else {
                fence_proxy_async_smem();
                issue(j, rec_next);
                nissued = j + 1;
                if (j + 1 < nproc) rec_next = N.rec[j + 1];
            }
        }
        pfail = __shfl_sync(0xffffffffu, pf, 0);
        rc = rcn;
        r2c = r2n;
        r2n = r2nn;
        Xn = Xnn;
        Xs = Xsn;
        if (++b == nbuf) {
            b = 0;
            ph ^= 1u;
        }
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = nissued > nbuf ? nissued - nbuf : 0; j < nissued; ++j)
            if (j < p.issue_end) mbar_wait_bounded(&full[j % nbuf], (uint32_t)((j / nbuf) & 1));
    }
    // totals out of tensor memory (every lane of the warp takes part in the loads)
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t sv[8], cv[8];
        tm_ld8(tbase + 8 * k, sv);
        tm_ld8(tbase + 32 + 8 * k, cv);
        tm_wait_ld();
        if (valid && wact) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int s = 2 * k + (u >> 1);           // 16-byte chunk slot of these two outputs
                const int o = m0 + ((s ^ l8) << 2) + 2 * (u & 1);
                const double v0 = (double)__uint_as_float(sv[2 * u]) - (double)__uint_as_float(cv[2 * u]);
                const double v1 = (double)__uint_as_float(sv[2 * u + 1]) - (double)__uint_as_float(cv[2 * u + 1]);
                if (o < m) p.y[q * m + o] = (bad || failed) ? nanv : v0;
                if (o + 1 < m) p.y[q * m + o + 1] = (bad || failed) ? nanv : v1;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(kTmCols) : "memory");
}

static cudaError_t launch_nodal_tmem(const EvalParams &p, cudaStream_t st) {
    const DevNodal &N = p.t.nod[p.form];
    const int buf = (int)((N.stage_bytes[DDSG_F32C] + 127) & ~127ll);
    const int nbuf = 128 + 3 * (int64_t)buf <= kSmemLimit ? 3 : 2;
    const int smem = 128 + nbuf * buf;
    const int64_t items = (p.n + kTmQB - 1) / kTmQB * (N.rs32 >> 5);   // (query tile, 32-output window)
    dim3 grid((unsigned)((items + 1) / 2));
    cudaError_t e = cudaFuncSetAttribute(eval_nodal_tmem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    eval_nodal_tmem_kernel<<<grid, kTmNT, smem, st>>>(p, buf, nbuf);
    return cudaGetLastError();
}

bool nodal_eligible(const DevTables &t, int precision, int form) {
    const DevNodal &N = t.nod[form];
    if (!N.ok || !N.vals) return false;
    const int64_t buf = (N.stage_bytes[precision] + 127) & ~127ll;
    return 128 + 2 * buf <= kSmemLimit;
}

template <int PREC, int MC, int GR>
static cudaError_t launch_nodal(const EvalParams &p, cudaStream_t st) {
    constexpr int QB = NodShape<GR>::QB, NT = NodShape<GR>::NT;
    const DevNodal &N = p.t.nod[p.form];
    const int buf = (int)((N.stage_bytes[PREC] + 127) & ~127ll);
    const int nbuf = 128 + 3 * (int64_t)buf <= kSmemLimit ? 3 : 2;
    const int smem = 128 + nbuf * buf;
    const int rs = PREC == DDSG_F64 ? p.t.mp64 : N.rs32;
    const int per_block = MC * GR;
    dim3 grid((unsigned)((p.n + QB - 1) / QB), (unsigned)((rs + per_block - 1) / per_block));
    cudaError_t e = cudaFuncSetAttribute(eval_nodal_kernel<PREC, MC, GR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    eval_nodal_kernel<PREC, MC, GR><<<grid, NT, smem, st>>>(p, buf, nbuf);
    return cudaGetLastError();
}

template <int GR>
static cudaError_t launch_nodal_f32x2(const EvalParams &p, cudaStream_t st) {
    constexpr int QB = NodShape<GR>::QB, NT = NodShape<GR>::NT;
    const DevNodal &N = p.t.nod[p.form];
    const int buf = (int)((N.stage_bytes[DDSG_F32C] + 127) & ~127ll);
    const int nbuf = 128 + 3 * (int64_t)buf <= kSmemLimit ? 3 : 2;
    const int smem = 128 + nbuf * buf;
    dim3 grid((unsigned)((p.n + QB - 1) / QB), (unsigned)((N.rs32 + 32 * GR - 1) / (32 * GR)));
    cudaError_t e = cudaFuncSetAttribute(eval_nodal_f32x2_kernel<GR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    eval_nodal_f32x2_kernel<GR><<<grid, NT, smem, st>>>(p, buf, nbuf);
    return cudaGetLastError();
}

cudaError_t launch_eval_nodal_tmem(const EvalParams &p, cudaStream_t st) { return launch_nodal_tmem(p, st); }

cudaError_t launch_eval_nodal(const EvalParams &p, int precision, int mc, cudaStream_t st) {
    const DevNodal &N = p.t.nod[p.form];
    if (precision == DDSG_F32C) {
        if (mc == 32 && N.rs32 % 32 == 0)
            return N.rs32 > 32 ? launch_nodal_f32x2<2>(p, st) : launch_nodal_f32x2<1>(p, st);
        if (mc == 8) return launch_nodal<DDSG_F32C, 8, 1>(p, st);
        return launch_nodal<DDSG_F32C, 16, 1>(p, st);
    }
    if (mc == 4) return launch_nodal<DDSG_F64, 4, 1>(p, st);
    if (mc == 16) return launch_nodal<DDSG_F64, 16, 1>(p, st);
    return launch_nodal<DDSG_F64, 8, 1>(p, st);
}

}  // namespace ddsg
