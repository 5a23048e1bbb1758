/*
 * ddsg.h -- C ABI of libddsg: batched evaluation of a cut-HDMR adaptive
 * sparse-grid ("DDSG") interpolant on one GB300 GPU (sm_103a).
 *
 * Method: Eftekhari & Scheidegger, "High-Dimensional Dynamic Stochastic Model
 * Representation", arXiv 2202.06555.
 *   - sparse grids, hat basis, surpluses, refinement:   Sec. 3.1, eq. 3.1-3.8
 *   - cut-HDMR and its telescopic components:           Sec. 3.2, eq. ddsg2.2.5-2.2.6
 *   - DDSG approximation:                               Sec. 3.3, eq. 3.16
 *   - vectorized evaluation f(x) = a(x)^T b:            Sec. 4.1, eq. 4.2
 *   - IRBC model residual (Euler equations):            Sec. 2.1, eq. model1-model2
 *
 * Conventions shared by every call
 *   d        state dimension; m number of outputs (policy components).
 *   Domain   physical box [lo_i, hi_i]; a coordinate maps to [0,1] by
 *            (x - lo)/(hi - lo) and is clamped to [0,1] (clamps are counted).
 *   Basis    boundary-augmented hats (Sec. 3.1, "augmenting the basis"):
 *            level 1: constant 1 (node 1/2, index 1);
 *            level 2: nodes 0 and 1 (index 0 and 2), phi = max(0, 1 - |2x - i|);
 *            level l >= 3: nodes i/2^(l-1), i odd, phi = max(0, 1 - |2^(l-1)x - i|).
 *            Level constraint of a level-L grid: sum_j (l_j - 1) <= L - 1 (eq. 3.5).
 *   Points   a component of k dimensions stores per point k levels (uint8)
 *            and k indices (uint32); arrays are point-major: levels[p*k + j].
 *   Order    canonical point order is (level sum, level tuple, index tuple),
 *            lexicographic; refinement appends new points in that order.
 *   Memory   pointers named *_dev are device pointers the caller owns (e.g.
 *            torch tensors); pointers named *_host are host arrays, copied
 *            before the call returns. The handle owns every device table.
 *   Streams  calls taking a cudaStream_t are asynchronous on that stream.
 *   Errors   every call returns DDSG_OK (0) or a negative DDSG_ERR_* code and
 *            stores a message readable by ddsg_last_error() (thread-local).
 *            Kernels never trap: bad inputs become NaN outputs and counters.
 */
#ifndef DDSG_H
#define DDSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ddsg_stream_t; /* == cudaStream_t; NULL = legacy default stream */
typedef struct hdmr hdmr_t;                /* opaque handle */

enum {
    DDSG_OK = 0,
    DDSG_ERR_ARG = -1,     /* invalid argument (sizes, ranges, NULL)                */
    DDSG_ERR_OOM = -2,     /* device or host allocation failed                      */
    DDSG_ERR_CUDA = -3,    /* a CUDA runtime call failed                            */
    DDSG_ERR_STATE = -4,   /* call out of order (e.g. eval before hierarchize)      */
    DDSG_ERR_TABLE = -5,   /* invalid grid table (range, duplicate, level sum)      */
    DDSG_ERR_TIMEOUT = -6, /* a bounded device wait gave up                         */
    DDSG_ERR_NUMERIC = -7  /* non-finite values where finite ones are required      */
};

enum { DDSG_F64 = 0, DDSG_F32C = 1 };            /* arithmetic of hdmr_eval           */
enum { DDSG_FORM_PAPER = 0, DDSG_FORM_SLICEFREE = 1 };

#define DDSG_KMAX 8        /* most dimensions of one component                       */
#define DDSG_LMAX 24       /* highest 1D level                                        */

/* Last error message of the calling thread ("" if none). */
const char *ddsg_last_error(void);
/* Library version string. */
const char *ddsg_version(void);

/*
 * ddsg_inject_alloc_failure -- TEST ONLY (no paper counterpart), process-wide:
 * after `skip` more device allocations by the library succeed, the next
 * `count` fail as on an exhausted device (nothing is allocated; the call that
 * needed the memory returns DDSG_ERR_OOM). count = 0 turns the switch off.
 * Every entry point leaves its handle consistent after such a failure: the
 * same call succeeds once memory is available again. Negative arguments are
 * DDSG_ERR_ARG. Makes no CUDA call.
 */
int ddsg_inject_alloc_failure(int skip, int count);

/*
 * Checked builds (the library compiled with -DDDSG_CHECKED; no paper
 * counterpart): the bounds-checked stand-in for a memory sanitizer. Every
 * table index a kernel derives from the grid tables (cell offset, directory
 * slot, device row against its component's rows, staged block, dimension,
 * point and component ids) is tested before the access it guards; a failed
 * test sets one bit per site in a process-wide check word and skips the access
 * (the result of that query is wrong, nothing is touched out of bounds).
 * ddsg_checked_build() is 1 in such a build, 0 otherwise.
 * ddsg_take_check_word reads and clears the word: bit 0 cell, 1 slot, 2 row,
 * 3 stage, 4 dimension, 5 point, 6 component (always 0 in release builds).
 * Synchronous.
 */
int ddsg_checked_build(void);
int ddsg_take_check_word(uint64_t *word);

/*
 * hdmr_create -- new empty expansion (Sec. 4.2, Alg. 2 inputs: anchor, order).
 *   d >= 1, m >= 1, 0 <= order <= DDSG_KMAX.
 *   anchor_host, lo_host, hi_host: length d, physical units, lo < hi.
 *   The slice-free form additionally needs the anchor at the domain centre
 *   (canonical 1/2, the level-1 node); hdmr_eval refuses it otherwise.
 *   Makes no CUDA call: the handle binds to the current CUDA device at its
 *   first GPU use (hdmr_hierarchize, hdmr_reserve, hdmr_stats) and must be
 *   used on that device afterwards.
 */
int hdmr_create(int d, int m, int order, const double *anchor_host, const double *lo_host,
                const double *hi_host, hdmr_t **out);
int hdmr_destroy(hdmr_t *h);

/*
 * hdmr_add_component -- append the grid of component u = dims (eq. ddsg2.2.6:
 * it will interpolate the cut function f(anchor \ x_u)).
 *   k = |u| in [0, order]; dims_host strictly ascending in [0, d); k = 0 is the
 *   empty component (npts must be 1, levels/indices may be NULL).
 *   levels_host/indices_host: npts*k. Checked: level in [1, DDSG_LMAX], index
 *   valid for its level, no duplicate point, u not already present.
 *   Returns the component id (insertion order) in *comp_id.
 *   The b coefficients of eq. 4.2 are computed over the accepted set as given
 *   when the tables are first uploaded (hdmr_hierarchize). A set that is not
 *   downward closed (e.g. one full-dimensional sparse grid alone) is valid
 *   for the paper form; the slice-free form needs closure.
 */
int hdmr_add_component(hdmr_t *h, int k, const int32_t *dims_host, int64_t npts,
                       const uint8_t *levels_host, const uint32_t *indices_host, int32_t *comp_id);

/* Same, with the regular level-`level` grid of eq. 3.5 generated by the library. */
int hdmr_add_regular_component(hdmr_t *h, int k, const int32_t *dims_host, int level,
                               int32_t *comp_id);

/* Sizes: number of components and total points. */
int hdmr_num_components(const hdmr_t *h, int32_t *ncomp, int64_t *npts_total);

/*
 * hdmr_component_info -- k, dims (DDSG_KMAX entries, unused = -1), number of
 * points and the offset of its first point in the concatenated point order
 * used by hdmr_hierarchize.
 */
int hdmr_component_info(const hdmr_t *h, int32_t comp, int32_t *k, int32_t *dims_host,
                        int64_t *npts, int64_t *first_point);

/*
 * hdmr_component_points -- levels/indices (count*k) and physical node
 * coordinates (count*k, on the component's dims) of points
 * [first, first+count) of component comp. Any output may be NULL. The caller
 * evaluates f at these nodes with the other coordinates at the anchor
 * (the cut points of eq. ddsg2.2.6).
 */
int hdmr_component_points(const hdmr_t *h, int32_t comp, int64_t first, int64_t count,
                          uint8_t *levels_host, uint32_t *indices_host, double *coords_host);

/*
 * hdmr_hierarchize -- surpluses of every point (Sec. 3.1; "surplus = value
 * minus the coarser interpolant"), computed on the GPU in FP64:
 *   alpha_p = v_p - sum_{q in G_u, levelsum(q) < levelsum(p)} alpha_q phi_q(x_p),
 * layer by layer in increasing level sum, all components in one launch.
 *   values_dev: device, npts_total*m FP64, components in id order, points in
 *   table order (the layout hdmr_component_info's first_point describes).
 *   Also refreshes the FP32 copy of the surpluses used by DDSG_F32C.
 * Synchronous with respect to the host on return of the table upload only;
 * the hierarchization itself is asynchronous on `stream`.
 */
int hdmr_hierarchize(hdmr_t *h, const double *values_dev, ddsg_stream_t stream);

/*
 * hdmr_refine -- one adaptive refinement sweep of every component (eq. 3.8):
 * a point is significant if ||alpha_p||_inf > eps_gamma; each child of a
 * significant point, in each dimension of its component, is added when its
 * level tuple satisfies sum(l-1) <= max_level-1 and it is not yet present.
 *   strict = 0: a child of at least one significant parent is added.
 *   strict = 1: a child is dropped if any present parent of it is not
 *               significant (the stricter reading of Sec. 3.1, where finer
 *               points inside the support of a rejected point are left out).
 * New points are appended per component in canonical order; *n_new = total.
 * Needs hierarchized surpluses (reads them back, synchronizing `stream`).
 * A non-finite surplus (from a non-finite value given to hdmr_hierarchize)
 * is DDSG_ERR_NUMERIC, naming the component, point and output; nothing is
 * added then.
 * The new points need values before the next hdmr_hierarchize.
 */
int hdmr_refine(hdmr_t *h, double eps_gamma, int max_level, int strict, int64_t *n_new,
                ddsg_stream_t stream);

/*
 * Checkpoint / resume (no paper counterpart). hdmr_save writes the expansion
 * (domain, anchor, every component's points, the FP64 surpluses) to one
 * versioned binary file with a checksum; it needs a hierarchized handle and
 * synchronizes the device. hdmr_load recreates a hierarchized handle on the
 * current device from such a file (no values or hierarchization needed);
 * a missing, foreign, truncated or corrupt file is DDSG_ERR_ARG. Results of
 * hdmr_eval on the loaded handle equal the saved one's bit for bit.
 * hdmr_shape returns d, m, order and the anchor / lo / hi host arrays (d each;
 * any output may be NULL).
 */
int hdmr_save(const hdmr_t *h, const char *path);
int hdmr_load(const char *path, hdmr_t **out);
int hdmr_shape(const hdmr_t *h, int32_t *d, int32_t *m, int32_t *order, double *anchor_host,
               double *lo_host, double *hi_host);

/*
 * hdmr_quadrature -- the integral over [0,1]^k of every component interpolant
 * (eq. 3.7; canonical coordinates): q_dev[c*m + o] = sum over the points of
 * component c of alpha_p[o] * prod_j (1, 1/4 or 2^-(l-1) for level 1, 2, l >= 3).
 * These feed the expansion criterion (eq. 3.18) and the active dimension
 * selection (eq. 3.19). q_dev: device, ncomp*m FP64. FP64, asynchronous on
 * `stream`; the handle must be hierarchized.
 */
int hdmr_quadrature(hdmr_t *h, double *q_dev, ddsg_stream_t stream);

/*
 * hdmr_expansion_norms -- the criteria of Alg. 2 for the components of order k,
 * from the component integrals of hdmr_quadrature:
 *   qf_host (ncomp*m, nullable): the cut-HDMR component integrals
 *     Qf_u = sum over v subset of u of (-1)^(|u|-|v|) Q_v (every subset of every
 *     component must itself be a component: DDSG_ERR_ARG otherwise);
 *   eta_host (ncomp, nullable): eq. 3.19, eta_u = ||Qf_u||_2 / ||sum_{|v|<=k-1} Qf_v||_2
 *     for |u| = k, NaN for the other components;
 *   *rho_all (nullable): eq. 3.18 over all components of order k;
 *   *rho_kept (nullable): the same over those kept (eta_u > eps_eta; all of them
 *     when k = 1).
 * FP64; synchronous on `stream`; allocates ncomp*m doubles of device scratch.
 */
int hdmr_expansion_norms(hdmr_t *h, int k, double eps_eta, double *qf_host, double *eta_host, double *rho_all,
                         double *rho_kept, ddsg_stream_t stream);

/* Copy FP64 surpluses of all points to the host (npts_total*m). Synchronous. */
int hdmr_get_surpluses(const hdmr_t *h, double *alpha_host, ddsg_stream_t stream);

/* b coefficients of eq. 4.2 (one per component, id order), computed on the
 * host: b_v = sum over accepted u containing v of (-1)^(|u|-|v|). No CUDA call. */
int hdmr_get_b(const hdmr_t *h, double *b_host);

/*
 * hdmr_eval -- f(x) for n query points (the vectorized DDSG interpolation of
 * Sec. 4.1).
 *   x_dev: device, n*d FP64, physical units, row-major.
 *   y_dev: device, n*m FP64, row-major (written).
 *   precision: DDSG_F64 -- FP64 basis products and sums;
 *              DDSG_F32C -- FP32 surpluses and basis values, FP32 products,
 *              compensated (Kahan) accumulation, result rounded to FP64.
 *   form: DDSG_FORM_PAPER -- y = sum_v b_v s_v(x), eq. 4.2 (components with
 *              b_v = 0 skipped);
 *         DDSG_FORM_SLICEFREE -- y = sum_u (sum of the points of G_u whose
 *              levels are all >= 2); equal to the paper form when the anchor
 *              is the level-1 node and every slice {l_j = 1, j in u\w} of G_u
 *              equals G_w (true for grids built by hdmr_refine from cut
 *              values); it avoids the cancellation of large |b_v|.
 *   hash_dev (nullable, n uint64) / count_dev (nullable, n int32): XOR of the
 *   point keys / number of summed points with phi_p(x) > 0 in exact
 *   arithmetic (the active set). Key of point (l, i) of component c:
 *     z = c; for j < k: z = mix(z ^ (l_j << 40) ^ i_j); key = mix(z + 0x9E3779B97F4A7C15)
 *   with mix the SplitMix64 finalizer (Steele, Lea & Flood 2014):
 *     z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB; z ^= z>>31.
 *   Non-finite coordinates give NaN rows (counted in hdmr_stats).
 *   The slice-free form needs the anchor at the domain centre and a
 *   downward-closed component set (DDSG_ERR_ARG otherwise).
 *   Asynchronous on `stream`. Uses a handle-owned workspace that grows on
 *   demand (cudaMalloc): call hdmr_reserve first to make it capture-safe.
 */
int hdmr_eval(hdmr_t *h, int64_t n, const double *x_dev, double *y_dev, int precision, int form,
              uint64_t *hash_dev, int32_t *count_dev, ddsg_stream_t stream);

/*
 * Evaluation kernel choice (the batching schedule). kernel 0 = tile kernel
 * (1D bases of a component staged once per dimension and level), kernel 1 =
 * per-tuple kernel, kernels 2-4 = tile kernels whose component surplus blocks
 * are staged into shared memory by TMA bulk copies, three-deep (one, two or
 * three warp groups per query; need every evaluated component's block to fit
 * the staging buffer, k <= 2 and levels <= 15; refused otherwise), kernel 5 =
 * the staged nodal-slab kernel: each component's interpolant stored by node
 * values along one dimension per cell of the other (hdmr_nodal_info), two node
 * rows per slab level and query instead of one surplus row per level tuple
 * (k <= 2; its tables are planned and uploaded on first use, which allocates).
 * Kernel 5 has no per-point active set: a call with hash_dev or count_dev
 * evaluates with kernel 0. mc = outputs per thread and pass (0 = the
 * heuristic: smallest compiled chunk >= m; kernel 5: 32 = the FP32 layout of
 * 32-output windows read in a bank-conflict-free rotated order). hdmr_autotune
 * times every compiled pair on the caller's queries (x_dev, n; y_dev is
 * scratch output) and keeps the fastest for (precision, form); *best_ms
 * (nullable) gets its time. Autotuning runs the evaluation about 40 times:
 * tune on a representative subset of the queries.
 */
int hdmr_set_eval_config(hdmr_t *h, int precision, int form, int kernel, int mc);
int hdmr_get_eval_config(const hdmr_t *h, int precision, int form, int *kernel, int *mc);
int hdmr_autotune(hdmr_t *h, int64_t n, const double *x_dev, double *y_dev, int precision,
                  int form, ddsg_stream_t stream, double *best_ms);

/*
 * hdmr_nodal_info -- the nodal-slab tables of evaluation kernel 5 for `form`
 * (no paper counterpart: a change of basis of the component interpolants of
 * Sec. 3.1). Plans and uploads them if they are not built yet (allocates).
 * *eligible: 1 if kernel 5 can hold these tables; *rows: node rows stored;
 * *rows_per_query: node rows a query uniformly distributed in the domain reads,
 * summed over the components (the kernel's work per query). Pointers nullable.
 */
int hdmr_nodal_info(hdmr_t *h, int form, int32_t *eligible, int64_t *rows, double *rows_per_query);

/*
 * hdmr_eval_noalloc -- hdmr_eval (no hash/count outputs) that allocates no
 * device memory. The paper has no counterpart; this exists for callers that
 * must not allocate while they evaluate: frameworks that own all device
 * memory through their own pool or run under a fixed memory cap, and
 * latency-critical loops where an allocation would stall or fail. hdmr_eval
 * grows a handle workspace with cudaMalloc; this call instead uses one
 * file-scope static device array of 16 MiB (2^21 words), which every GPU that
 * loads the library keeps reserved until the process exits.
 *   n must not exceed hdmr_eval_noalloc_capacity(d) (= floor(2^22 / (2d + 1)):
 *   n*d coordinates plus n flags); larger batches are refused with
 *   DDSG_ERR_ARG before anything runs -- split them.
 *   The first call on a device looks up the array's device address there
 *   (cudaGetSymbolAddress, once per device); a call with n = 0 does only
 *   that. Under lazy module loading (CUDA's default) this first call is also
 *   when the 16 MiB are committed on the device, so make it while setting up:
 *   before any stream capture begins and before a memory cap applies.
 *   Launches are traced like hdmr_eval's (DDSG_K_ENCODE, DDSG_K_EVAL); waits
 *   that give up count in hdmr_stats and hdmr_check reports them, and the
 *   handle's hdmr_set_fault_injection switch applies here too.
 *   All calls on a device share the array and it keeps the last call's
 *   contents (each call overwrites all it reads). Calls whose kernels overlap
 *   on the GPU race on it: serialize them on one stream.
 *   The handle must be hierarchized. Asynchronous on `stream`.
 */
int hdmr_eval_noalloc(hdmr_t *h, int64_t n, const double *x_dev, double *y_dev, int precision,
                      int form, ddsg_stream_t stream);
/* Largest n hdmr_eval_noalloc accepts for dimension d (0 if d < 1). */
int64_t hdmr_eval_noalloc_capacity(int d);

/*
 * hdmr_eval_graph -- hdmr_eval (no hash/count outputs) replayed from a CUDA
 * graph. Each time-iteration step of Sec. 2.2 (and each Newton iteration inside
 * it) evaluates the same policy at same-sized state sets, so the launches of
 * one evaluation (query encoding and the fused all-component kernel) are
 * captured once and replayed. The handle caches one executable graph for the
 * last (n, x_dev, y_dev, precision, form, schedule); a call with any of them
 * different, or after the grid, the hierarchized tables' storage or the
 * workspace size changed, captures again (allocations happen before capture).
 * The graph reads x_dev and writes y_dev by address: refill x_dev in place
 * between calls. The replay runs on a handle-owned stream ordered after the
 * work already queued on `stream`, and work queued on `stream` afterwards runs
 * after it. Same results as hdmr_eval, bit for bit. Tracing counts each replay
 * under DDSG_K_GRAPH. Not thread-safe per handle (nor is any call).
 */
int hdmr_eval_graph(hdmr_t *h, int64_t n, const double *x_dev, double *y_dev, int precision,
                    int form, ddsg_stream_t stream);

/*
 * hdmr_set_fault_injection -- TEST ONLY (no paper counterpart): exercises the
 * failure path of the TMA-staged evaluation kernels without faulting anything.
 * From the processed component withhold_from on (-1: off, the default) the
 * kernel's producer thread issues no staging copies, so the bounded waits on
 * them (2^18 polls of mbarrier.try_wait, about one second) run out. A block that gives up writes
 * NaN for its queries and counts one timeout per warp in hdmr_stats (stats[2]);
 * the copies it did issue land before it exits and the context stays usable.
 * Applies to hdmr_eval, hdmr_eval_host, hdmr_eval_graph and hdmr_eval_noalloc of this handle
 * (not to the evaluations inside euler_residual / irbc_newton). Only kernels
 * 2-4 (hdmr_set_eval_config) stage; the others ignore the setting, which
 * persists until set back to -1.
 */
int hdmr_set_fault_injection(hdmr_t *h, int withhold_from);

/* Pre-size the eval workspace for up to n queries (no allocation in later evals). */
int hdmr_reserve(hdmr_t *h, int64_t n);

/*
 * hdmr_stats -- counters accumulated by hdmr_eval since the last reset:
 *   stats[0] = clamped coordinates, stats[1] = non-finite query rows,
 *   stats[2] = bounded device waits that gave up (staging copies that did not
 *   arrive in time; the affected outputs are invalid). stats_host holds 3.
 * Synchronizes `stream`. reset != 0 zeroes them afterwards.
 */
int hdmr_stats(hdmr_t *h, int64_t *stats_host, int reset, ddsg_stream_t stream);

/*
 * hdmr_check -- status of the evaluations queued so far: synchronizes `stream`
 * and returns DDSG_ERR_TIMEOUT if a staged evaluation kernel gave up a bounded
 * wait since the counter was last cleared (by this call or a hdmr_stats
 * reset): the queries of the blocks that gave up read NaN. The timeout
 * counter is cleared when it is reported. In a checked build it then returns
 * DDSG_ERR_TABLE (naming the sites) if any table index test failed since the
 * check word was last taken, and clears the word. DDSG_OK otherwise, and
 * before the handle's first GPU use.
 */
int hdmr_check(hdmr_t *h, ddsg_stream_t stream);

/*
 * hdmr_eval_host -- hdmr_eval with HOST buffers x_host (n*d) and y_host (n*m);
 * synchronizes `stream` before returning. Page-locked buffers are accessed by
 * the kernels through their mapped device addresses: the encoding kernel reads
 * x_host and the evaluation kernel writes y_host directly, so the transfers
 * overlap the computation. Other host memory goes through a handle-owned
 * device buffer with a copy before (x) or after (y) the evaluation. The whole
 * round trip is the end-to-end cost of one call.
 */
int hdmr_eval_host(hdmr_t *h, int64_t n, const double *x_host, double *y_host, int precision,
                   int form, ddsg_stream_t stream);

/*
 * Kernel timing (tracing). While enabled, every kernel the handle launches is
 * bracketed by CUDA events recorded on its launching stream; hdmr_profile_read
 * waits for them and returns, per kernel kind, the summed device milliseconds
 * and the number of launches since the last reset. Do not enable while the
 * stream is being captured into a CUDA graph.
 */
enum {
    DDSG_K_ENCODE = 0,   /* query encoding (clamp, fixed point)   */
    DDSG_K_EVAL = 1,     /* interpolant evaluation               */
    DDSG_K_HIER = 2,     /* hierarchization                      */
    DDSG_K_CONVERT = 3,  /* FP64 -> FP32 surplus copy            */
    DDSG_K_COPY = 4,     /* host<->device copies of hdmr_eval_host */
    DDSG_K_GRAPH = 5,    /* one graph replay of hdmr_eval_graph   */
    DDSG_NKINDS = 8
};
int hdmr_profile(hdmr_t *h, int enable);
int hdmr_profile_read(hdmr_t *h, double *ms_host /* DDSG_NKINDS */,
                      int64_t *launches_host /* DDSG_NKINDS */, int reset);

/* ------------------------------------------------------------------------
 * IRBC model step (Sec. 2.1): Euler equations (eq. model1), aggregate
 * resource constraint (eq. model2), productivity law of motion (eq.
 * law_of_motion); expectation by a degree-3 monomial rule over the N+1
 * shocks (2(N+1) nodes +-sqrt(N+1) e_i, equal weights).
 * ------------------------------------------------------------------------ */
typedef struct irbc irbc_t;

/* Table 1 values (beta, alpha, delta, sigma, rho, phi) and the aggregate
 * productivity A = (1 - beta (1 - delta)) / (alpha beta); N countries. */
typedef struct {
    int32_t N;
    double beta, alpha, delta, sigma, rho, phi, A;
} irbc_params_t;

/* New model; gamma_host, tau_host (length N, Table 1's gamma_j and tau_j) are
 * copied. Makes no CUDA call. */
int irbc_create(const irbc_params_t *prm, const double *gamma_host, const double *tau_host,
                irbc_t **out);
/* New model calibrated as in Table 1: the caller gives N, the curvature offset
 * a_gamma (0.25 in Table 1), beta, alpha, delta, sigma, rho and phi; the
 * library derives A = (1 - beta (1 - delta)) / (alpha beta), gamma_j = a_gamma +
 * 0.75 (j - 1) / (N - 1) (a_gamma when N = 1) and tau_j = A^(1 / gamma_j).
 * DDSG_ERR_ARG for N outside [1, 4096] or beta, alpha outside (0, 1), delta
 * outside [0, 1), a_gamma <= 0. Makes no CUDA call. */
int irbc_create_table1(int N, double a_gamma, double beta, double alpha, double delta, double sigma,
                       double rho, double phi, irbc_t **out);
/* The model's parameters (prm), gamma_j and tau_j (length N); pointers nullable. */
int irbc_get_params(const irbc_t *model, irbc_params_t *prm, double *gamma_host, double *tau_host);
int irbc_destroy(irbc_t *model);

/*
 * euler_residual -- residuals at ns states for the policy guess.
 *   policy: hierarchized hdmr_t over x = (a_1..a_N, k_1..k_N) (d = 2N) with
 *           m = N+1 outputs (k'_1..k'_N, lambda); its domain clamps next states.
 *   states_dev: ns x 2N, guess_dev: ns x (N+1) (k', lambda), resid_dev: ns x (N+1)
 *           (rows j < N: eq. model1 of country j+1; row N: eq. model2); with
 *           irbc_set_irreversible the widths are 2N+1 (see there).
 *   jac_dev (nullable): ns x (N+1) x (N+1), row-major d resid / d guess, from the
 *           hat slopes (right derivative at kinks, zero where k'_i is clamped)
 *           and the chain rule. Needs every policy component that holds a k_i
 *           to hold at most one a_j (any order-2 expansion qualifies;
 *           DDSG_ERR_ARG otherwise); a column whose component has more active
 *           points than the kernel's term buffer (48) is NaN.
 *   euler_err_dev (nullable): ns x 2, unit-free Euler error per state:
 *           max_j |beta E_j / (lambda (1 + phi g_j)) - 1| and |resource| / sum_j Y_j.
 *   precision/form: those of hdmr_eval for the policy interpolation; residual
 *   arithmetic is FP64. Asynchronous on `stream`; uses a model workspace
 *   (cudaMalloc, up to ~2 GiB; states are processed in chunks).
 */
int euler_residual(irbc_t *model, hdmr_t *policy, int64_t ns, const double *states_dev,
                   const double *guess_dev, double *resid_dev, double *jac_dev,
                   double *euler_err_dev, int precision, int form, ddsg_stream_t stream);

/*
 * irbc_set_node_mode -- how euler_residual (and so irbc_newton) obtains the
 * policy at the 2(N+1) monomial-rule nodes of each state.
 *   DDSG_IRBC_NODES_ALL (default): the interpolant at every node, as written.
 *   DDSG_IRBC_NODES_DELTA: the nodes of one state differ only in a' (footnote
 *     to Sec. 2.1's expectation: country node +-i shocks a'_i alone, the two
 *     global nodes shock every a'). The policy is interpolated at the no-shock
 *     state and the two global nodes; at country node +-i it is the no-shock
 *     policy plus, for each component holding a_i, that component at the
 *     shocked a'_i minus it at the no-shock a'_i (exact by the additive cut-HDMR
 *     form; differences are rounding only). Needs no assumption on the
 *     component set. About N times less interpolation work. The changes are
 *     kept in the evaluation precision and the residual's node sums expand
 *     around the no-shock policy: FP64 no-shock and global-node terms plus
 *     sums of the changes (FP32 with DDSG_F32C).
 */
enum { DDSG_IRBC_NODES_ALL = 0, DDSG_IRBC_NODES_DELTA = 1 };

/*
 * irbc_set_irreversible -- switch the model to the non-smooth IRBC of Sec. 2.1
 * (irreversible investment, eq. modelkink1). The policy then maps x = (a, k)
 * to (k'_1..k'_N, mu_1..mu_N, lambda) (m = 2N+1; guesses and solutions the
 * same). Residual rows: j < N the Euler equations with -mu_j today and
 * (1 - delta) mu'_j inside the expectation; N + j the complementarity
 * 0 <= mu_j _|_ k'_j - (1 - delta) k_j >= 0 as the Fischer-Burmeister
 * equation mu + I - sqrt(mu^2 + I^2) = 0 (its Jacobian row uses a generalized
 * derivative, 1 - 1/sqrt 2 per argument at mu = I = 0); 2N the resource
 * constraint. Newton is then a semismooth Newton method. Needs 2N+1 <= 165.
 */
int irbc_set_irreversible(irbc_t *model, int on);
int irbc_set_node_mode(irbc_t *model, int mode);

/* Batched dense LU with partial pivoting: dx = -A^{-1} r for ns systems of
 * size n (A_dev ns x n x n row-major FP64, r_dev/dx_dev ns x n), to FP64
 * accuracy. Factored in FP32 and refined in FP64 against A (iterative
 * refinement); a system the FP32 factors cannot refine (condition number
 * near 1/u_32 or beyond) is factored again in FP64. status_dev[s]: 0 solved,
 * 1 solved by the FP64 factorization, 2 exactly singular pivot (dx_dev[s]
 * undefined). n <= 165. */
int irbc_lu_solve(int n, int64_t ns, const double *A_dev, const double *r_dev, double *dx_dev,
                  int32_t *status_dev, ddsg_stream_t stream);

/*
 * irbc_newton -- per-state FP64 Newton on the residuals of euler_residual:
 * analytic Jacobian, LU solve, backtracking on ||r||_2 (halving up to 11
 * times). sol_dev (ns x m: m = N+1, or 2N+1 with irreversible investment)
 * holds the initial guess and receives the solution. Stops a state when
 * ||r||_inf <= tol. Outputs (nullable): iters_dev, status_dev (0 converged,
 * 1 max_it reached, 2 singular Jacobian), resnorm_dev (final ||r||_inf).
 * Each step is solved as irbc_lu_solve does, refined to FP64 accuracy with
 * precision DDSG_F64 and to 2^-30 of the step with DDSG_F32C (whose
 * Jacobian carries FP32 derivative sums). The line search evaluates its trial
 * points with the Jacobian, which the next iteration reuses; converged states
 * leave the working set. A state's iterates do not depend on the other
 * states of the batch. Synchronizes `stream` between iterations. Its device
 * buffers (about ns * m^2 * 8 bytes for the Jacobians) stay on the model for
 * later calls and are freed by irbc_destroy.
 */
int irbc_newton(irbc_t *model, hdmr_t *policy, int64_t ns, const double *states_dev,
                double *sol_dev, int max_it, double tol, int32_t *iters_dev, int32_t *status_dev,
                double *resnorm_dev, int precision, int form, ddsg_stream_t stream);

/* Kernel timing of a model (as hdmr_profile/hdmr_profile_read). Kinds:
 * 0 next-state queries, 1 policy interpolation, 2 residual sums, 3 Jacobian,
 * 4 LU solves, 5 Newton norms/trial points, 6 node-shortcut deltas; arrays
 * hold DDSG_NKINDS entries. */
int irbc_profile(irbc_t *model, int enable);
int irbc_profile_read(irbc_t *model, double *ms_host, int64_t *launches_host, int reset);

/* ------------------------------------------------------------------------
 * Warm-start network (no paper counterpart: the paper solves every grid
 * point from the previous policy; this MLP only proposes Newton initial
 * guesses). Hidden layers use the exact-erf GELU, the last layer is linear;
 * inputs are normalized as (x - in_shift) * in_scale and the network is
 * trained (mean squared error) on targets normalized as
 * (y - out_shift) * out_scale. GEMMs are hand-written BF16 tensor-core
 * kernels (tcgen05.mma with TMA operand tiles and FP32 accumulators in tensor
 * memory); master weights and Adam (beta 0.9/0.999, eps 1e-8) are FP32.
 * ------------------------------------------------------------------------ */
typedef struct mlp mlp_t;

/* sizes: nlayers+1 widths (input .. output). params_host (nullable): packed
 * FP32 parameters, per layer W (out x in, row-major) then b; NULL draws
 * W ~ U(-1/sqrt(in), 1/sqrt(in)) from SplitMix64(seed) and b = 0. No CUDA call. */
int mlp_create(int nlayers, const int32_t *sizes, const float *params_host, uint64_t seed,
               mlp_t **out);
int mlp_destroy(mlp_t *net);
/* Affine normalizations (host arrays; set before the first GPU call). */
int mlp_set_normalization(mlp_t *net, const double *in_shift, const double *in_scale,
                          const double *out_shift, const double *out_scale);
/* One Adam step on B rows: x_dev B x in (FP64), y_dev B x out (FP64).
 * loss_dev (nullable, device FP64) receives the batch loss. Asynchronous. */
int mlp_train_step(mlp_t *net, int64_t B, const double *x_dev, const double *y_dev, float lr,
                   double *loss_dev, ddsg_stream_t stream);
/* y_dev (B x out, FP64, physical units) = network(x_dev). Asynchronous. */
int mlp_infer(mlp_t *net, int64_t B, const double *x_dev, double *y_dev, ddsg_stream_t stream);
/* Packed parameters / gradients of the last train step (FP32, host). Synchronous. */
int64_t mlp_num_params(const mlp_t *net);
int mlp_get_params(mlp_t *net, float *host);
int mlp_get_grads(mlp_t *net, float *host);

/*
 * mlp_save / mlp_load -- checkpoint / resume of a network (no paper
 * counterpart): layer sizes, normalization, FP32 master weights, both Adam
 * moments and the Adam step count, in one versioned file ending in an FNV-1a
 * checksum. A loaded network continues training where the saved one stopped:
 * the same further steps give the same weights bit for bit. mlp_save
 * synchronizes the device; mlp_load makes no CUDA call (the network binds at
 * its first GPU use). A missing, foreign, truncated or corrupt file is
 * DDSG_ERR_ARG. mlp_shape: the layer count and the L+1 widths (sizes_host
 * nullable).
 */
int mlp_save(mlp_t *net, const char *path);
int mlp_load(const char *path, mlp_t **out);
int mlp_shape(const mlp_t *net, int32_t *nlayers, int32_t *sizes_host);
/* Kernel timing: kinds 0 forward GEMMs, 1 backward GEMMs, 2 loss/normalization, 3 Adam. */
int mlp_profile(mlp_t *net, int enable);
/*
 * ddsg_probe_fma -- measured FMA throughput of the current device (no paper
 * counterpart): the peak the evaluation kernels' ALU rooflines divide by.
 * kind 0: FP64 fma; 1: FP32 fmaf; 2: paired FP32 (fma.rn.f32x2). Runs 8
 * independent chains per thread on 8 blocks of 256 threads per SM, times the
 * second of two launches with CUDA events; *tflops = 2 flops per FMA / time,
 * *ms (nullable) the launch time. Synchronous; allocates 16 bytes.
 */
int ddsg_probe_fma(int kind, double *tflops, double *ms);

/*
 * mlp_check -- status of the network's tensor-core GEMMs since the last check
 * (no paper counterpart). Every mbarrier wait in them is bounded; a wait that
 * gives up leaves that GEMM's output tile unwritten and is recorded here.
 * Synchronizes the device; returns DDSG_ERR_TIMEOUT (and clears the record) if
 * any wait gave up, else DDSG_OK.
 */
int mlp_check(mlp_t *net);
int mlp_profile_read(mlp_t *net, double *ms_host, int64_t *launches_host, int reset);

#ifdef __cplusplus
}
#endif
#endif /* DDSG_H */
