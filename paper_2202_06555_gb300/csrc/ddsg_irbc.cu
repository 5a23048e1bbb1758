// ddsg_irbc.cu -- smooth and non-smooth IRBC model step on the GPU (Sec. 2.1 of
// the paper): Euler-equation residuals (eq. model1; eq. modelkink1 with
// irreversible investment) and the aggregate resource constraint (eq. model2)
// at a batch of states, with the expectation taken by a degree-3 monomial rule
// over the 2(N+1) shocks; an analytic Jacobian; a batched mixed-precision LU;
// and a damped Newton solve.
//
// Pipeline of one residual sweep (states processed in chunks that fit the
// model's workspace):
//   irbc_queries_kernel   next state x' = (a', k') at every (state, node)
//                         (eq. law_of_motion), encoded into the evaluation
//                         kernels' dimension-major fixed-point layout;
//                         node shortcut: irbc_queries3_kernel, only the
//                         no-shock state and the two global-shock nodes;
//   launch_eval           the policy interpolant at those queries (FP64 or F32C);
//   irbc_delta_kernel     node shortcut: each country node's policy change from
//                         the no-shock policy, from the components holding a_i;
//   irbc_residual_kernel  one block per state: node sums (FP64; with the node
//                         shortcut FP64 no-shock terms plus sums of the changes),
//                         residuals, Euler errors and the Jacobian's border and
//                         diagonal pieces;
//   irbc_jacobian_kernel  one block per state: d r_j / d k'_i through the
//                         components holding dim N+i, whose a-coordinate (if
//                         any) takes only three values over the nodes.
// irbc_newton iterates residual, LU (lu_mixed_kernel: FP32 factors refined in
// FP64, lu_solve_kernel in FP64 for the rest) and a backtracking line search
// over a working set from which converged states leave.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cmath>

#include <algorithm>
#include <string>
#include <vector>

#include "ddsg_alloc.h"
#include "ddsg_eval.cuh"
#include "ddsg_internal.h"
#include "ddsg_tables.h"

using namespace ddsg;

namespace {

struct IrbcDev {
    int N;
    int m;      // policy outputs: N + 1 (k', lambda) or 2N + 1 (k', mu, lambda)
    int irr;    // irreversible investment (eq. modelkink1): mu_j and a complementarity row
    double beta, alpha, delta, sigma, rho, phi, A;
    double shk_p, shk_m;   // exp(+sigma sqrt(N + 1)), exp(-sigma sqrt(N + 1))
    const double *gamma, *tau;
};

// Encode one physical coordinate exactly like the query encoder.
__device__ __forceinline__ uint64_t encode_coord(double v, double lo, double span, bool &bad,
                                                 unsigned long long &clamps) {
    double c = (v - lo) / span;
    if (!isfinite(v) || !isfinite(c)) {
        bad = true;
        return X_NAN;
    }
    if (c < 0.0) { c = 0.0; ++clamps; }
    if (c > 1.0) { c = 1.0; ++clamps; }
    const double yv = c * 4611686018427387904.0;
    uint64_t Xv = (uint64_t)yv;
    if ((double)Xv != yv) Xv |= 1ull;
    return Xv;
}

// Next-period productivity of country j at the three distinct node values:
// no shock on j (e0), +sqrt(N+1) (ep), -sqrt(N+1) (em), i.e. exp(rho ln a + sigma (e_j + e))
// taken as a^rho times the model's constant shock factor exp(sigma (e_j + e)).
__device__ __forceinline__ void next_a3(const IrbcDev &P, double a, double &e0, double &ep, double &em) {
    e0 = exp(P.rho * log(a));
    ep = e0 * P.shk_p;
    em = e0 * P.shk_m;
}

// Which of the three values node q gives to country j (nodes 2i / 2i+1 shock
// country i by +/-; nodes 2N / 2N+1 shock every country through the global shock).
__device__ __forceinline__ int node_variant(int q, int j, int N) {
    if (q == 2 * j || q == 2 * N) return 1;
    if (q == 2 * j + 1 || q == 2 * N + 1) return 2;
    return 0;
}

// One thread per (state, dimension): writes that coordinate for all nq nodes.
__global__ void irbc_queries_kernel(IrbcDev P, int64_t ns, const double *__restrict__ states,
                                    const double *__restrict__ guess, const double *__restrict__ lo,
                                    const double *__restrict__ span, uint64_t *__restrict__ X,
                                    int32_t *__restrict__ flags, unsigned long long *__restrict__ stats) {
    const int N = P.N, d = 2 * N, m = P.m, nq = 2 * (N + 1);
    const int64_t Q = ns * nq;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long clamps = 0;
    if (idx < ns * d) {
        const int64_t s = idx / d;
        const int dim = (int)(idx - s * d);
        bool bad = false;
        uint64_t *Xrow = X + (int64_t)dim * Q + s * nq;
        if (dim < N) {
            double v[3];
            next_a3(P, states[s * d + dim], v[0], v[1], v[2]);
            uint64_t e[3];
            const unsigned long long mult[3] = {(unsigned long long)(nq - 4), 2ull, 2ull};  // nodes per value
            for (int t = 0; t < 3; ++t) {
                unsigned long long c1 = 0;
                e[t] = encode_coord(v[t], lo[dim], span[dim], bad, c1);
                clamps += c1 * mult[t];
            }
            for (int q = 0; q < nq; ++q) Xrow[q] = e[node_variant(q, dim, N)];
            if (!isfinite(states[s * d + N + dim])) bad = true;
        } else {
            const uint64_t e = encode_coord(guess[s * m + dim - N], lo[dim], span[dim], bad, clamps);
            clamps *= (unsigned long long)nq;
            for (int q = 0; q < nq; ++q) Xrow[q] = e;
            if (dim == d - 1)
                for (int o = N; o < m; ++o)
                    if (!isfinite(guess[s * m + o])) bad = true;
        }
        if (bad)
            for (int q = 0; q < nq; ++q) flags[s * nq + q] = 1;
    }
    for (int o = 16; o > 0; o >>= 1) clamps += __shfl_down_sync(0xffffffffu, clamps, o);
    if ((threadIdx.x & 31) == 0 && clamps) atomicAdd(&stats[0], clamps);
}

// Per state (block): residuals, Euler errors and Jacobian pieces. Rows j < N:
// the Euler equation of country j (eq. model1; with irreversible investment
// eq. modelkink1, which adds -mu_j today and (1 - delta) mu'_j inside the
// expectation); rows N + j (irreversible only): the complementarity
// 0 <= mu_j _|_ k'_j - (1 - delta) k_j >= 0 as the Fischer-Burmeister equation
// mu + I - sqrt(mu^2 + I^2) = 0; row m - 1: the resource constraint (eq. model2).
// aux (per state, 7 x N): S1, SM, the diagonal part of d r_j / d k'_j, the three
// a'_j values (no shock, +, -), k'_j^(alpha-1); the Jacobian kernel reads them.
// Block: RES_THREADS at most (N rounded up to a warp), threads over countries j.
// The next-period policy at the nodes comes as NodePolicy<DELTA, W>: all 2(N+1)
// node rows (y), or with the node shortcut the no-shock and global-shock rows
// (y3) plus each country node's change from the no-shock row (dY, in W).
constexpr int RES_THREADS = 256;

template <bool DELTA, class W>
struct NodePolicy {
    const double *y;    // all nodes: nq rows of m per state
    const double *y3;   // shortcut: no shock, every country +, every country -
    const W *dY;        // shortcut: 2N rows of m per state, node 2i + u (u = 0: +, 1: -)
};

template <bool DELTA, class W>
__global__ void __launch_bounds__(RES_THREADS) irbc_residual_kernel(IrbcDev P, int64_t s0, int64_t nsc,
                                                            const double *__restrict__ states,
                                                            const double *__restrict__ guess,
                                                            const NodePolicy<DELTA, W> pol,
                                                            double *__restrict__ resid,
                                                            double *__restrict__ err,
                                                            double *__restrict__ jac,
                                                            double *__restrict__ aux) {
    const int N = P.N, d = 2 * N, m = P.m, nq = 2 * (N + 1);
    const int L = m - 1;                      // lambda's position in the policy
    const int64_t sl = blockIdx.x;           // state within the chunk
    const int64_t s = s0 + sl;                // global state
    const double *a = states + s * d;
    const double *k = states + s * d + N;
    const double *kp = guess + s * m;
    const double lam = guess[s * m + L];
    const double w = 1.0 / (double)nq;
    const double *ys = DELTA ? nullptr : pol.y + sl * nq * (int64_t)m;
    const double *yb = DELTA ? pol.y3 + sl * 3 * (int64_t)m : nullptr;   // no shock
    const double *ygp = yb ? yb + m : nullptr, *ygm = yb ? yb + 2 * m : nullptr;   // global +, -
    const W *dY = DELTA ? pol.dY + sl * 2 * N * (int64_t)m : nullptr;
    double res = 0.0, ysum = 0.0, emax = 0.0, dlam = 0.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // sum over the nodes of lambda', shared by every country: once per state
    // (threads over the nodes, then the warps' partials in warp order; with the
    // shortcut the sum of the country nodes' changes, added to the FP64 terms)
    __shared__ double red[4][RES_THREADS / 32];
    __shared__ double lsum_sh, dl_sh;
    {
        double ls = 0.0;
        if constexpr (DELTA) {
            W lw = (W)0;
            for (int c = threadIdx.x; c < 2 * N; c += blockDim.x) lw += dY[(int64_t)c * m + L];
            ls = (double)lw;
        } else {
            for (int q = threadIdx.x; q < nq; q += blockDim.x) ls += ys[(int64_t)q * m + L];
        }
        for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
        if (lane == 0) red[0][warp] = ls;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int wq = 0; wq < (int)(blockDim.x >> 5); ++wq) t += red[0][wq];
            if constexpr (DELTA) {
                dl_sh = t;   // sum of the country nodes' lambda' changes
                t += (double)(2 * N) * yb[L] + ygp[L] + ygm[L];
            }
            lsum_sh = t;
        }
        __syncthreads();
    }
    const double Lall = lsum_sh;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double e3[3];
        next_a3(P, a[j], e3[0], e3[1], e3[2]);
        const double g1 = kp[j] / k[j] - 1.0;
        const double kpa = pow(kp[j], P.alpha - 1.0);
        const double mu = P.irr ? guess[s * m + N + j] : 0.0;
        // node sums with the node weight w and the node-independent factors taken
        // out (FP64 is GB300's slow unit: one reciprocal of k'_j per j, none per
        // node). With r = k''_j / k'_j (g2 = r - 1):
        //   M_q = a' A alpha k'^(alpha-1) + (1 - delta) + phi/2 (r^2 - 1),
        //   d/dk'_j [lambda' M_q] at fixed next-period policy
        //       = lambda' (a' A alpha (alpha-1) k'^(alpha-1) - phi r^2) / k'_j,
        // the a'-dependent constants taken once per shock variant.
        const double ikp = 1.0 / kp[j];
        const double cA = P.A * P.alpha * kpa;
        const double hphi = 0.5 * P.phi;
        const double mb0 = e3[0] * cA + ((1.0 - P.delta) - hphi), mb1 = e3[1] * cA + ((1.0 - P.delta) - hphi),
                     mb2 = e3[2] * cA + ((1.0 - P.delta) - hphi);
        const double db0 = e3[0] * cA * (P.alpha - 1.0), db1 = e3[1] * cA * (P.alpha - 1.0),
                     db2 = e3[2] * cA * (P.alpha - 1.0);
        // M_q = hphi r^2 + mb_v and d/dk'_j [lambda' M_q] = (db_v - 2 hphi r^2) lambda' / k'_j with
        // r = k''_j / k'_j and v the node's a'_j value, so every node sum follows from
        // A1 = sum lambda' k'', A2 = sum lambda' k''^2, K2 = sum k''^2 and the sums of
        // lambda' per value (value 1: the nodes 2j and 2N, value 2: 2j+1 and 2N+1,
        // value 0: the others; their total Lall is the state's): three FP64
        // operations per node (four with the Jacobian) instead of ten.
        double A1 = 0.0, A2 = 0.0, K2 = 0.0, Ms = 0.0, L1, L2;
        if constexpr (DELTA) {
            // country node c: k'' = kb + dk_c, lambda' = lb + dl_c. The sums of the
            // changes run in W (FP32 with F32C), the no-shock and global terms in FP64:
            //   A1 = 2N lb kb + lb S1 + kb Dl + P1 + globals,
            //   A2 = 2N lb kb^2 + 2 lb kb S1 + lb S2 + kb^2 Dl + 2 kb P1 + P2 + globals,
            //   K2 = 2N kb^2 + 2 kb S1 + S2 + globals,
            // S1 = sum dk, S2 = sum dk^2, P1 = sum dl dk, P2 = sum dl dk^2, Dl = sum dl.
            W s1 = (W)0, s2 = (W)0, p1 = (W)0, p2 = (W)0, sm = (W)0;
#pragma unroll 4
            for (int c = 0; c < 2 * N; ++c) {
                const W dk = dY[(int64_t)c * m + j];
                const W dl = dY[(int64_t)c * m + L];
                const W t = dl * dk;
                s1 += dk;
                p1 += t;
                s2 = fma(dk, dk, s2);
                p2 = fma(t, dk, p2);
                if (P.irr) sm += dY[(int64_t)c * m + N + j];
            }
            const double kb = yb[j], lb = yb[L], n2 = (double)(2 * N);
            const double S1 = (double)s1, S2 = (double)s2, P1 = (double)p1, P2 = (double)p2, Dl = dl_sh;
            const double kp_ = ygp[j], km_ = ygm[j], lp_ = ygp[L], lm_ = ygm[L];
            A1 = n2 * lb * kb + lb * S1 + kb * Dl + P1 + (lp_ * kp_ + lm_ * km_);
            A2 = n2 * lb * kb * kb + 2.0 * lb * kb * S1 + lb * S2 + kb * kb * Dl + 2.0 * kb * P1 + P2 +
                 (lp_ * kp_ * kp_ + lm_ * km_ * km_);
            if (jac) K2 = n2 * kb * kb + 2.0 * kb * S1 + S2 + (kp_ * kp_ + km_ * km_);
            if (P.irr) Ms = n2 * yb[N + j] + (double)sm + (ygp[N + j] + ygm[N + j]);
            L1 = (lb + (double)dY[(int64_t)(2 * j) * m + L]) + lp_;
            L2 = (lb + (double)dY[(int64_t)(2 * j + 1) * m + L]) + lm_;
        } else {
#pragma unroll 4
            for (int q = 0; q < nq; ++q) {
                const double kpp = ys[(int64_t)q * m + j];
                const double lamp = ys[(int64_t)q * m + L];
                const double t = lamp * kpp;
                A1 += t;
                A2 = fma(t, kpp, A2);
                if (jac) K2 = fma(kpp, kpp, K2);
                if (P.irr) Ms += ys[(int64_t)q * m + N + j];
            }
            L1 = ys[(int64_t)(2 * j) * m + L] + ys[(int64_t)(2 * N) * m + L];
            L2 = ys[(int64_t)(2 * j + 1) * m + L] + ys[(int64_t)(2 * N + 1) * m + L];
        }
        const double L0 = Lall - L1 - L2;
        const double ikp2 = ikp * ikp;
        const double Es = fma(hphi * ikp2, A2, fma(mb0, L0, fma(mb1, L1, mb2 * L2)));
        const double S1s = ikp * A1;
        const double SMs = fma(hphi * ikp2, K2, fma(mb0, (double)(nq - 4), 2.0 * (mb1 + mb2)));
        const double Ds = fma(-2.0 * hphi * ikp2, A2, fma(db0, L0, fma(db1, L1, db2 * L2)));
        // E = sum_q w lambda' M_q (- (1 - delta) w mu'_j when irreversible);
        // S1 = sum_q w lambda' phi (g2 + 1) / k'_j, SM = sum_q w M_q,
        // Dd = d/dk'_j of sum_q w lambda' M_q at fixed next-period policy
        const double E = w * Es - (P.irr ? w * (1.0 - P.delta) * Ms : 0.0);
        const double S1 = w * P.phi * ikp * S1s, SM = w * SMs, Dd = w * ikp * Ds;
        const double lhs = lam * (1.0 + P.phi * g1) - mu;
        resid[s * m + j] = lhs - P.beta * E;
        emax = fmax(emax, fabs(P.beta * E / lhs - 1.0));
        const double inv = kp[j] - (1.0 - P.delta) * k[j];
        const double rr = sqrt(mu * mu + inv * inv);
        if (P.irr) resid[s * m + N + j] = mu + inv - rr;
        const double Y = a[j] * P.A * pow(k[j], P.alpha);
        ysum += Y;
        const double cj = pow(lam / P.tau[j], -P.gamma[j]);
        res += Y + k[j] * ((1.0 - P.delta) - 0.5 * P.phi * g1 * g1) - kp[j] - cj;
        if (jac) {
            double *J = jac + s * (int64_t)m * m;
            J[(int64_t)j * m + L] = 1.0 + P.phi * g1;        // d r_j / d lambda
            J[(int64_t)L * m + j] = -(1.0 + P.phi * g1);     // d resource / d k'_j
            dlam += P.gamma[j] * cj / lam;                   // d resource / d lambda
            if (P.irr) {
                for (int i = 0; i < N; ++i) J[(int64_t)j * m + N + i] = i == j ? -1.0 : 0.0;   // d r_j / d mu_i
                J[(int64_t)L * m + N + j] = 0.0;                                              // d resource / d mu_j
                // complementarity row: a generalized derivative of FB, (1 - 1/sqrt 2) at the kink
                double *Jr = J + (int64_t)(N + j) * m;
                for (int c = 0; c < m; ++c) Jr[c] = 0.0;
                const double ga = rr > 0.0 ? 1.0 - mu / rr : 1.0 - 0.70710678118654752;
                const double gb = rr > 0.0 ? 1.0 - inv / rr : 1.0 - 0.70710678118654752;
                Jr[j] = gb;
                Jr[N + j] = ga;
            }
            double *ax = aux + sl * 7 * (int64_t)N;
            ax[0 * N + j] = S1;
            ax[1 * N + j] = SM;
            ax[2 * N + j] = lam * P.phi / k[j] - P.beta * Dd;  // diagonal part of d r_j / d k'_j
            ax[3 * N + j] = e3[0];
            ax[4 * N + j] = e3[1];
            ax[5 * N + j] = e3[2];
            ax[6 * N + j] = kpa;
        }
    }
    // block reductions (sum / max) in a fixed order: warp butterflies, then the
    // warps' partials in warp order (any block size that is a multiple of 32)
    for (int o = 16; o > 0; o >>= 1) {
        res += __shfl_xor_sync(0xffffffffu, res, o);
        ysum += __shfl_xor_sync(0xffffffffu, ysum, o);
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        dlam += __shfl_xor_sync(0xffffffffu, dlam, o);
    }
    if (lane == 0) {
        red[0][warp] = res;
        red[1][warp] = ysum;
        red[2][warp] = emax;
        red[3][warp] = dlam;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
        for (int wq = 0; wq < (int)(blockDim.x >> 5); ++wq) {
            r0 += red[0][wq];
            r1 += red[1][wq];
            r2 = fmax(r2, red[2][wq]);
            r3 += red[3][wq];
        }
        resid[s * m + L] = r0;
        if (err) {
            err[s * 2 + 0] = r2;
            err[s * 2 + 1] = fabs(r0) / r1;
        }
        if (jac) jac[s * (int64_t)m * m + (int64_t)L * m + L] = r3;
    }
}

// Right derivative in c of hat (l, cell containing X): +-2^(l-1), 0 at level 1.
__device__ __forceinline__ double dhat(uint64_t X, int l, uint32_t &cell) {
    if (l == 1) { cell = 0; return 0.0; }
    if (l == 2) {
        cell = X >= (1ull << 61) ? 1u : 0u;
        return cell ? 2.0 : -2.0;
    }
    const int sh = 64 - l;
    uint64_t c = X >> sh;
    const uint64_t nmax = (1ull << (l - 2)) - 1;
    if (c > nmax) c = nmax;
    cell = (uint32_t)c;
    const uint64_t F = X - (c << sh);
    const double mag = (double)(1ull << (l - 1));
    return F < (1ull << (sh - 1)) ? mag : -mag;
}

// Terms of d p(x)/d x_dpos for one component at coordinates Xd (one per
// component dimension; position dpos is the differentiated one): appends
// (device row, weight) pairs, the weight holding coef (b or 1) and 1/span,
// multiplied in W.
// Returns the number of terms, or -1 if there were more than cap.
// Surplus table and row stride of each evaluation precision: FP64 rows, or
// the FP32 rows that F32C multiplies in FP32.
template <int PREC>
struct DeltaT;
template <>
struct DeltaT<DDSG_F64> {
    using W = double;
    static __device__ __forceinline__ const double *alpha(const DevTables &t) { return t.alpha64; }
    static __device__ __forceinline__ int stride(const DevTables &t) { return t.mp64; }
};
template <>
struct DeltaT<DDSG_F32C> {
    using W = float;
    static __device__ __forceinline__ const float *alpha(const DevTables &t) { return t.alpha32; }
    static __device__ __forceinline__ int stride(const DevTables &t) { return t.mp32; }
};

// (device row, weight) of one term; the weight in the precision the terms are summed in
template <class W>
struct DTerm { int32_t row; W w; };

template <class W>
__device__ int comp_dterms(const DevTables &t, const DevComp &cd, int tb, int dpos, const uint64_t *Xd,
                           W scale, DTerm<W> *out, int cap) {
    int n = 0;
    for (int ti = tb; ti < cd.tup_end; ++ti) {
        const DevTup tu = t.tups[ti];
        uint32_t off = 0;
        W wt = scale;
        bool act = true;
        for (int j = 0; j < cd.k; ++j) {
            const int l = tu.lev[j];
            if (j == dpos) {
                uint32_t cell;
                const double sl = dhat(Xd[j], l, cell);
                if (sl == 0.0) { act = false; break; }
                wt *= (W)sl;   // +-2^(l-1): exact
                off = off * (j == 1 ? tu.nc1 : ncells(l)) + cell;
            } else {
                Basis1D o;
                if (!basis1d(Xd[j], l, o)) { act = false; break; }
                wt *= basis_val<W>(o);
                off = off * (j == 1 ? tu.nc1 : ncells(l)) + o.cell;
            }
        }
        if (!act) continue;
        const int32_t row = tuple_row_at(tu, off, t.slots, t.S, cd.row_begin, cd.row_end);
        if (row < 0) continue;
        if (n == cap) return -1;
        out[n].row = row;
        out[n].w = wt;
        ++n;
    }
    return n;
}

constexpr int DT_CAP = 48;

// Jacobian columns d r_j / d k'_i (j < N) of each state, one block per state.
// k'_i enters the next-period policy through every component holding dim
// N+i. For such a component u the coordinates of u at a node are the base
// ones (no shock on u's country, if any) except at the nodes shocking u's
// a-dimension (country c: nodes 2c, 2N get a'_c at +, nodes 2c+1, 2N+1 at -):
// its slope in k'_i takes at most three values over the 2(N+1) nodes, and the
// node sum splits into the base sum (total minus the four shocked nodes) plus
// those four. Components holding k_i and more than one a-dimension make the
// column NaN (the host refuses such sets), and so does a column whose
// derivative terms do not fit the shared pool.
// Phase 1: a thread per (column i, component) group finds the derivative terms
// (device row, weight) of each of its up to three variants and appends them to
// a shared pool. Phase 2: a warp per column, lanes over the outputs j, sums
// weight x surplus row over each variant's terms, so every term's row is read
// coalesced, and adds the node factors of output j.
// PREC: F64 sums the derivative terms in FP64 from the FP64 surpluses; F32C
// multiplies and sums them in FP32 from the FP32 surpluses (Newton needs the
// Jacobian only to FP32 accuracy; the residual itself stays FP64).
constexpr int JAC_THREADS = 256;
constexpr int JAC_KJ = 6;   // outputs per lane: N <= 32 * JAC_KJ = 192

// A node policy value in W. For FP32 the conversion is done on the integer
// units from the IEEE-754 fields (sign, exponent rebiased, significand cut to
// 23 bits: rounding toward zero, within one FP32 ulp, which the Jacobian
// tolerates); zeros, values outside FP32's normal range, infinities and NaN
// take the hardware conversion. GB300's FP64 units (conversions included) are
// its slow ones.
template <class W>
__device__ __forceinline__ W to_w(double x);
template <>
__device__ __forceinline__ double to_w<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_w<float>(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff) - 1023 + 127;   // FP32 biased exponent
    if (ex < 1 || ex > 254) return (float)x;
    const uint32_t f = (uint32_t)(b >> 32) & 0x80000000u;
    return __uint_as_float(f | ((uint32_t)ex << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
}

// FP32 -> FP64 on the integer units (exact for every value: normal FP32 values
// from their fields, the others through the hardware conversion). GB300's FP64
// pipe runs conversions too, at 16 cycles per warp instruction.
__device__ __forceinline__ double widen_f32(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t ex = (b >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu) return (double)x;
    return __longlong_as_double((long long)(((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(ex + 896u) << 52) |
                                            ((uint64_t)(b & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return widen_f32(x); }

struct JGroup {
    int32_t i, ctry, nv, off[3], cnt[3];
    double dPN[3];
};

template <int PREC, bool DELTA>
__global__ void __launch_bounds__(JAC_THREADS) irbc_jacobian_kernel(IrbcDev P, int64_t s0, int64_t nsc,
                                                                   DevTables t, int form,
                                                                   const int32_t *__restrict__ koff,
                                                                   const int32_t *__restrict__ kids,
                                                                   const double *__restrict__ lo,
                                                                   const double *__restrict__ span,
                                                                   const double *__restrict__ guess,
                                                                   const NodePolicy<DELTA, typename DeltaT<PREC>::W> pol,
                                                                   const double *__restrict__ aux,
                                                                   double *__restrict__ jac, int pool_cap) {
    using W = typename DeltaT<PREC>::W;
    const int N = P.N, m = P.m, nq = 2 * (N + 1);
    const int L = m - 1;   // lambda's position in the policy
    const int64_t sl = blockIdx.x;   // state within the chunk (grid.x: no 65535 limit)
    const int64_t s = s0 + sl;
    const bool paper = form == DDSG_FORM_PAPER;
    const double *kp = guess + s * m;
    const double *ax = aux + sl * 7 * (int64_t)N;
    // node q's policy at output o: stored, or (shortcut) no-shock + change / global rows
    const double *ys = DELTA ? nullptr : pol.y + sl * nq * (int64_t)m;
    const double *y3s = DELTA ? pol.y3 + sl * 3 * (int64_t)m : nullptr;
    const W *dYs = DELTA ? pol.dY + sl * 2 * N * (int64_t)m : nullptr;
    auto node64 = [&](int q, int o) -> double {   // global nodes (q >= 2N) or all-node mode
        if constexpr (DELTA) return y3s[(int64_t)(q - 2 * N + 1) * m + o];
        else return ys[(int64_t)q * m + o];
    };
    auto nodew = [&](int q, int o) -> W {         // country nodes, in W
        if constexpr (DELTA) return to_w<W>(y3s[o]) + dYs[(int64_t)q * m + o];
        else return to_w<W>(ys[(int64_t)q * m + o]);
    };
    double *J = jac + s * (int64_t)m * m;
    const double w = 1.0 / (double)nq;
    const W *alpha = DeltaT<PREC>::alpha(t);
    const int mp = DeltaT<PREC>::stride(t);
    const int G = koff[N];
    extern __shared__ float4 jac_raw[];
    JGroup *grp = reinterpret_cast<JGroup *>(jac_raw);
    int32_t *colstate = reinterpret_cast<int32_t *>(grp + G);   // 0 normal, 1 clamped, 2 NaN
    // per output j, in W: S1, SM, 1/k'_j, A alpha k'^(alpha-1), and s1, sM at the
    // two global-shock nodes 2N (+) and 2N+1 (-), which every column shares
    W *oj = reinterpret_cast<W *>(reinterpret_cast<unsigned char *>(jac_raw) +
                                  ((sizeof(JGroup) * G + sizeof(int32_t) * N + 15) & ~(size_t)15));
    W *oS1 = oj, *oSM = oj + N, *oik = oj + 2 * N, *ocA = oj + 3 * N;
    W *os1p = oj + 4 * N, *osMp = oj + 5 * N, *os1m = oj + 6 * N, *osMm = oj + 7 * N;
    // a'_j at no shock / + / -, and (node shortcut) the no-shock k''_j, in W
    W *oa0 = oj + 8 * N, *oap = oj + 9 * N, *oam = oj + 10 * N, *okb = oj + 11 * N;
    // per country j: k'_j and the three a'_j values (no shock, +, -) encoded once
    uint64_t *Xk = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(oj) +
                                                ((sizeof(W) * 12 * N + 15) & ~(size_t)15));
    uint64_t *Xa = Xk + N;   // Xa[3 j + v]
    DTerm<W> *pool = reinterpret_cast<DTerm<W> *>(Xk + 4 * N);
    __shared__ int cursor;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) cursor = 0;
    for (int i = tid; i < N; i += JAC_THREADS) {
        // k'_i in canonical units; clamped (or at the top face) -> zero derivative
        const double ck = (kp[i] - lo[N + i]) / span[N + i];
        colstate[i] = (ck >= 0.0 && ck < 1.0) ? 0 : 1;
        const int j = i;
        const double ik = 1.0 / kp[j], cA = P.A * P.alpha * ax[6 * N + j];
        oS1[j] = (W)ax[0 * N + j];
        oSM[j] = (W)ax[1 * N + j];
        oik[j] = (W)ik;
        ocA[j] = (W)cA;
        oa0[j] = (W)ax[3 * N + j];
        oap[j] = (W)ax[4 * N + j];
        oam[j] = (W)ax[5 * N + j];
        okb[j] = DELTA ? (W)y3s[j] : (W)0;
        {
            bool bd = false;
            unsigned long long cl = 0;
            Xk[j] = encode_coord(kp[j], lo[N + j], span[N + j], bd, cl);
            for (int v = 0; v < 3; ++v) Xa[3 * j + v] = encode_coord(ax[(3 + v) * N + j], lo[j], span[j], bd, cl);
        }
        for (int u = 0; u < 2; ++u) {
            const int q = 2 * N + u;   // global node: every a' shocked, variant 1 (+) or 2 (-)
            const double kpp = node64(q, j), lamp = node64(q, L);
            const double g2 = kpp * ik - 1.0;
            const double s1 = w * lamp * P.phi * (g2 + 1.0) * ik;
            const double sM = w * (ax[(4 + u) * N + j] * cA + (1.0 - P.delta) + 0.5 * P.phi * g2 * (g2 + 2.0));
            (u == 0 ? os1p : os1m)[j] = (W)s1;
            (u == 0 ? osMp : osMm)[j] = (W)sM;
        }
    }
    __syncthreads();
    // phase 1: the terms of every (column, component) group
    for (int g = tid; g < G; g += JAC_THREADS) {
        int lo_i = 0, hi_i = N;   // column i: koff[i] <= g < koff[i + 1]
        while (hi_i - lo_i > 1) {
            const int mid = (lo_i + hi_i) >> 1;
            if (koff[mid] <= g) lo_i = mid; else hi_i = mid;
        }
        const int i = lo_i, dk = N + i;
        JGroup gr;
        gr.i = i;
        gr.ctry = -1;
        gr.nv = 0;
        for (int v = 0; v < 3; ++v) { gr.off[v] = 0; gr.cnt[v] = 0; gr.dPN[v] = 0.0; }
        if (colstate[i] == 0 && comp_ok(t, kids[g], 2 * N)) {
            const DevComp &cd = t.comps[kids[g]];
            const double coef = paper ? cd.b : 1.0;
            if (coef != 0.0) {
                const int tb = paper ? cd.tup_begin : cd.tup_int;
                uint64_t Xd[KMAX];
                int dpos = 0, apos = -1, ctry = -1, na = 0;
                for (int j = 0; j < cd.k; ++j) {
                    const int dim = cd.dims[j];
                    if (dim == dk) {
                        dpos = j;
                        Xd[j] = Xk[i];
                    } else if (dim < N) {
                        apos = j;
                        ctry = dim;
                        ++na;
                        Xd[j] = Xa[3 * dim];
                    } else {
                        Xd[j] = Xk[dim - N];
                    }
                }
                const int nv = na == 0 ? 1 : 3;
                bool over = na > 1;
                DTerm<W> loc[DT_CAP];
                const W dscale = (W)(coef / span[dk]);
                for (int v = 0; v < nv && !over; ++v) {
                    if (v > 0) Xd[apos] = Xa[3 * ctry + v];
                    const int nt = comp_dterms<W>(t, cd, tb, dpos, Xd, dscale, loc, DT_CAP);
                    if (nt < 0) { over = true; break; }
                    const int off = atomicAdd(&cursor, nt);
                    if (off + nt > pool_cap) { over = true; break; }
                    W acc = (W)0;
                    for (int q = 0; q < nt; ++q) {
                        pool[off + q] = loc[q];
                        acc += loc[q].w * alpha[(int64_t)loc[q].row * mp + L];
                    }
                    gr.off[v] = off;
                    gr.cnt[v] = nt;
                    gr.dPN[v] = (double)acc;
                }
                if (over) {
                    colstate[i] = 2;
                } else {
                    gr.nv = nv;
                    gr.ctry = ctry;
                }
            }
        }
        grp[g] = gr;
    }
    __syncthreads();
    // phase 2: a warp per column i, lane outputs j = lane + 32 k; the node
    // factors and the column's sum over its groups in W (FP32 in the F32C
    // mode, like the derivative sums)
    const W beta = (W)P.beta, phi = (W)P.phi, ww = (W)w, omd = (W)(1.0 - P.delta);
    for (int i = warp; i < N; i += JAC_THREADS / 32) {
        const int cs = colstate[i];
        W acc[JAC_KJ];
#pragma unroll
        for (int kk = 0; kk < JAC_KJ; ++kk) acc[kk] = (W)0;
        if (cs == 0) {
            for (int g = koff[i]; g < koff[i + 1]; ++g) {
                const JGroup &gr = grp[g];
                const int nv = gr.nv;
                if (nv == 0) continue;
                // dPv[kk] = sum over the terms of variant v of weight x surplus row at output j
                // (dMv: at output N + j, the multiplier mu'_j of the irreversible model)
                W dP0[JAC_KJ], dP1[JAC_KJ], dP2[JAC_KJ], dM0[JAC_KJ], dM1[JAC_KJ], dM2[JAC_KJ];
                auto sumv = [&](int v, W (&oP)[JAC_KJ], W (&oM)[JAC_KJ]) {
                    W a1[JAC_KJ], a2[JAC_KJ];
#pragma unroll
                    for (int kk = 0; kk < JAC_KJ; ++kk) { a1[kk] = (W)0; a2[kk] = (W)0; }
                    for (int q = 0; q < gr.cnt[v]; ++q) {
                        const DTerm<W> tq = pool[gr.off[v] + q];
                        const W *row = alpha + (int64_t)tq.row * mp;
#pragma unroll
                        for (int kk = 0; kk < JAC_KJ; ++kk) {
                            const int j = lane + 32 * kk;
                            if (j < N) {
                                a1[kk] += tq.w * row[j];
                                if (P.irr) a2[kk] += tq.w * row[N + j];
                            }
                        }
                    }
#pragma unroll
                    for (int kk = 0; kk < JAC_KJ; ++kk) { oP[kk] = a1[kk]; oM[kk] = a2[kk]; }
                };
                sumv(0, dP0, dM0);
                if (nv == 3) {
                    sumv(1, dP1, dM1);
                    sumv(2, dP2, dM2);
                } else {
#pragma unroll
                    for (int kk = 0; kk < JAC_KJ; ++kk) dP1[kk] = dP2[kk] = dM1[kk] = dM2[kk] = (W)0;
                }
                const int ctry = gr.ctry;
                const W dPN0 = (W)gr.dPN[0], dPN1 = (W)gr.dPN[1], dPN2 = (W)gr.dPN[2];
                // lambda' at the country's two nodes (the same for every output)
                W lamq[2] = {(W)0, (W)0};
                if (nv == 3)
                    for (int u = 0; u < 2; ++u) lamq[u] = nodew(2 * ctry + u, L);
#pragma unroll
                for (int kk = 0; kk < JAC_KJ; ++kk) {
                    const int j = lane + 32 * kk;
                    if (j >= N) continue;
                    W v0;
                    if (nv == 1) {
                        v0 = -beta * (oS1[j] * dP0[kk] + oSM[j] * dPN0);
                    } else {
                        // the country nodes of u's country c: 2c (a'_c at +) and 2c+1 (-);
                        // a'_j moves there only when j = c. The global nodes come from oj.
                        const W ik = oik[j], cA = ocA[j];
                        W s1c[2], sMc[2];
                        for (int u = 0; u < 2; ++u) {
                            const int q = 2 * ctry + u;
                            const W kpp = DELTA ? okb[j] + dYs[(int64_t)q * m + j] : nodew(q, j);
                            const W lamp = lamq[u];
                            const W g2 = kpp * ik - (W)1;
                            const W ap = j == ctry ? (u == 0 ? oap[j] : oam[j]) : oa0[j];
                            s1c[u] = ww * lamp * phi * (g2 + (W)1) * ik;
                            sMc[u] = ww * (ap * cA + omd + (W)0.5 * phi * g2 * (g2 + (W)2));
                        }
                        const W s1P = s1c[0] + os1p[j], s1M = s1c[1] + os1m[j];
                        const W sMP = sMc[0] + osMp[j], sMM = sMc[1] + osMm[j];
                        const W s1b = oS1[j] - s1P - s1M, sMb = oSM[j] - sMP - sMM;
                        v0 = -beta * (s1b * dP0[kk] + s1P * dP1[kk] + s1M * dP2[kk] + sMb * dPN0 + sMP * dPN1 + sMM * dPN2);
                    }
                    if (P.irr) {
                        // (1 - delta) mu'_j inside the expectation: its slope in k'_i at the nodes
                        const W sumw = nv == 1 ? (W)nq * ww * dM0[kk]
                                               : ww * ((W)(nq - 4) * dM0[kk] + (W)2 * dM1[kk] + (W)2 * dM2[kk]);
                        v0 += beta * omd * sumw;
                    }
                    acc[kk] += v0;
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < JAC_KJ; ++kk) {
            const int j = lane + 32 * kk;
            if (j < N)
                J[(int64_t)j * m + i] = cs == 2 ? NAN : (j == i ? ax[2 * N + j] + to_f64(acc[kk]) : to_f64(acc[kk]));
        }
    }
}

// Shared memory of the Jacobian kernel: the groups, the column states, the
// per-country node factors and encoded coordinates, and a
// term pool sized for the most terms one state can collect (`terms`, from the
// tables' tuple counts), within kJacSmem bytes in all (a column whose terms
// do not fit is NaN). A pool sized to the tables lets several blocks share an SM.
constexpr size_t kJacSmem = 160 * 1024;

template <int PREC, bool DELTA>
static cudaError_t launch_jacobian_t(const IrbcDev &P, int64_t s0, int64_t nsc, const DevTables &t, int form,
                                     const int32_t *koff, const int32_t *kids, const double *lo, const double *span,
                                     const double *guess, const NodePolicy<DELTA, typename DeltaT<PREC>::W> &pol,
                                     const double *aux, double *jac, size_t smem, int cap, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(irbc_jacobian_kernel<PREC, DELTA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    irbc_jacobian_kernel<PREC, DELTA><<<(unsigned)nsc, JAC_THREADS, smem, st>>>(P, s0, nsc, t, form, koff, kids, lo, span,
                                                                             guess, pol, aux, jac, cap);
    return cudaGetLastError();
}

// y: all node rows, or (dY != null, the node shortcut) the 3 rows per state
// of the no-shock and global-shock queries, with dY the country nodes' changes
// (double for FP64, float for F32C)
static cudaError_t launch_jacobian(int precision, const IrbcDev &P, int64_t s0, int64_t nsc, const DevTables &t,
                                   int form, int G, int64_t terms, const int32_t *koff, const int32_t *kids,
                                   const double *lo, const double *span, const double *guess, const double *y,
                                   const void *dY, const double *aux, double *jac, cudaStream_t st) {
    const size_t wsz = precision == DDSG_F64 ? sizeof(double) : sizeof(float);
    const size_t fixed = ((sizeof(JGroup) * G + sizeof(int32_t) * P.N + 15) & ~(size_t)15) +
                         ((wsz * 12 * P.N + 15) & ~(size_t)15) + sizeof(uint64_t) * 4 * P.N;
    const size_t term = precision == DDSG_F64 ? sizeof(DTerm<double>) : sizeof(DTerm<float>);
    if (fixed + 64 * term > kJacSmem) return cudaErrorInvalidValue;
    const size_t cap = std::min<size_t>(std::max<int64_t>(terms, 1), (kJacSmem - fixed) / term);
    const size_t smem = fixed + cap * term;
    if (precision == DDSG_F64) {
        if (dY) {
            const NodePolicy<true, double> pol{nullptr, y, static_cast<const double *>(dY)};
            return launch_jacobian_t<DDSG_F64, true>(P, s0, nsc, t, form, koff, kids, lo, span, guess, pol, aux, jac,
                                                     smem, (int)cap, st);
        }
        const NodePolicy<false, double> pol{y, nullptr, nullptr};
        return launch_jacobian_t<DDSG_F64, false>(P, s0, nsc, t, form, koff, kids, lo, span, guess, pol, aux, jac, smem,
                                                  (int)cap, st);
    }
    if (dY) {
        const NodePolicy<true, float> pol{nullptr, y, static_cast<const float *>(dY)};
        return launch_jacobian_t<DDSG_F32C, true>(P, s0, nsc, t, form, koff, kids, lo, span, guess, pol, aux, jac, smem,
                                                  (int)cap, st);
    }
    const NodePolicy<false, float> pol{y, nullptr, nullptr};
    return launch_jacobian_t<DDSG_F32C, false>(P, s0, nsc, t, form, koff, kids, lo, span, guess, pol, aux, jac, smem,
                                               (int)cap, st);
}

// ---------------------------------------------------------------------------
// batched dense LU with partial pivoting (FP64, one block per system)
// ---------------------------------------------------------------------------

// (redo != 0: solve only the systems whose status is 3, the ones the mixed-precision
// kernel below could not refine, and set their status to 1 (solved here) or 2)
__global__ void __launch_bounds__(256) lu_solve_kernel(int n, int64_t ns, const double *__restrict__ Ag,
                                                       const double *__restrict__ bg, const int32_t *active,
                                                       double *__restrict__ xg, int32_t *__restrict__ status,
                                                       int redo) {
    extern __shared__ double sm[];
    double *A = sm;             // n x n
    double *b = sm + n * n;     // n
    __shared__ int piv;
    __shared__ double pval[256];
    __shared__ int pidx[256];
    const int64_t s = blockIdx.x;
    if (active && !active[s]) return;
    if (redo && status[s] != 3) return;
    const double *As = Ag + s * (int64_t)n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = As[e];
    for (int e = threadIdx.x; e < n; e += blockDim.x) b[e] = -bg[s * n + e];
    __syncthreads();
    bool singular = false;
    for (int c = 0; c < n; ++c) {
        // pivot: largest |A[r][c]| for r >= c (ties -> smallest r)
        double best = -1.0;
        int bi = c;
        for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
            const double v = fabs(A[r * n + c]);
            if (v > best) { best = v; bi = r; }
        }
        pval[threadIdx.x] = best;
        pidx[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                const double v2 = pval[threadIdx.x + o];
                const int i2 = pidx[threadIdx.x + o];
                if (v2 > pval[threadIdx.x] || (v2 == pval[threadIdx.x] && i2 < pidx[threadIdx.x])) {
                    pval[threadIdx.x] = v2;
                    pidx[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) piv = pidx[0];
        __syncthreads();
        const int p = piv;
        if (!(pval[0] > 0.0)) { singular = true; break; }
        if (p != c) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const double tmp = A[c * n + j];
                A[c * n + j] = A[p * n + j];
                A[p * n + j] = tmp;
            }
            if (threadIdx.x == 0) {
                const double tmp = b[c];
                b[c] = b[p];
                b[p] = tmp;
            }
        }
        __syncthreads();
        const double inv = 1.0 / A[c * n + c];
        for (int r = c + 1 + threadIdx.x; r < n; r += blockDim.x) {
            const double f = A[r * n + c] * inv;
            A[r * n + c] = f;
            for (int j = c + 1; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            b[r] -= f * b[c];
        }
        __syncthreads();
    }
    if (singular) {
        if (threadIdx.x == 0) status[s] = 2;
        return;
    }
    // back substitution (one thread; n is small)
    if (threadIdx.x == 0) {
        for (int r = n - 1; r >= 0; --r) {
            double acc = b[r];
            for (int j = r + 1; j < n; ++j) acc -= A[r * n + j] * b[j];
            b[r] = acc / A[r * n + r];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) xg[s * n + e] = b[e];
    if (redo && threadIdx.x == 0) status[s] = 1;
}

// ---------------------------------------------------------------------------
// batched LU, mixed precision: factor in FP32 in shared memory, refine in FP64
// (iterative refinement: solve with the FP32 factors, form the residual
// b - A x in FP64 from the original matrix, solve for the correction, repeat).
// On GB300 FP32 arithmetic is far faster than FP64 and the FP32 factors take
// half the shared memory (two systems per SM). Each system's refinement stops
// once the correction is below rtol of the solution (2^-46: FP64 accuracy). The
// corrections shrink by about cond(A) u_32 per step; a system whose
// correction stops halving, or that needs more than LUM_SOLVES solves
// (condition number near 1/u_32 or worse), gets status 3 and is solved again
// by the FP64 kernel above.
// ---------------------------------------------------------------------------

constexpr int LUM_THREADS = 256;
constexpr int LUM_WARPS = LUM_THREADS / 32;
constexpr int LUM_SOLVES = 12;  // first solve + up to 11 corrections (each must halve the last)

inline size_t lum_smem_bytes(int n) {
    const int ld = n | 1;
    const size_t a = ((size_t)n * ld * sizeof(float) + 15) & ~(size_t)15;
    return a + (size_t)n * (2 * sizeof(double) + sizeof(float) + sizeof(int));
}

// max over the block (every thread gets the result); red holds LUM_WARPS values
__device__ __forceinline__ double lum_block_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = red[0];
    for (int w = 1; w < LUM_WARPS; ++w) r = fmax(r, red[w]);
    return r;
}

// y <- U^-1 L^-1 y in place (L unit lower, U upper, both in A with stride ld):
// 32-row blocks, the diagonal block solved by warp 0 with shuffles, the rest
// of the rows updated by all threads.
__device__ __forceinline__ void lum_solve(const float *A, int ld, int n, float *y) {
    const int tid = threadIdx.x, lane = tid & 31;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int kb = min(32, n - k0);
        if (tid < 32) {
            float v = lane < kb ? y[k0 + lane] : 0.0f;
            for (int k = 0; k < kb; ++k) {
                const float yk = __shfl_sync(0xffffffffu, v, k);
                if (lane > k && lane < kb) v = fmaf(-A[(k0 + lane) * ld + k0 + k], yk, v);
            }
            if (lane < kb) y[k0 + lane] = v;
        }
        __syncthreads();
        for (int r = k0 + kb + tid; r < n; r += LUM_THREADS) {
            float acc = y[r];
            for (int k = 0; k < kb; ++k) acc = fmaf(-A[r * ld + k0 + k], y[k0 + k], acc);
            y[r] = acc;
        }
        __syncthreads();
    }
    for (int k1 = n; k1 > 0; k1 -= 32) {
        const int k0 = k1 > 32 ? k1 - 32 : 0, kb = k1 - k0;
        if (tid < 32) {
            float v = lane < kb ? y[k0 + lane] : 0.0f;
            for (int k = kb - 1; k >= 0; --k) {
                if (lane == k) v = v / A[(k0 + k) * ld + k0 + k];
                const float xk = __shfl_sync(0xffffffffu, v, k);
                if (lane < k) v = fmaf(-A[(k0 + lane) * ld + k0 + k], xk, v);
            }
            if (lane < kb) y[k0 + lane] = v;
        }
        __syncthreads();
        for (int r = tid; r < k0; r += LUM_THREADS) {
            float acc = y[r];
            for (int k = 0; k < kb; ++k) acc = fmaf(-A[r * ld + k0 + k], y[k0 + k], acc);
            y[r] = acc;
        }
        __syncthreads();
    }
}

// Rows c + 1 .. n - 1 of the factorization step at column c: a warp per row,
// lane entries j = c + 1 + lane + 32 kk, kk < NK, the pivot row's in registers.
template <int NK>
__device__ __forceinline__ void lum_update_rows(float *A, int ld, int n, int c, float inv, int lane, int warp) {
    float prow[NK];
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) {
        const int j = c + 1 + lane + 32 * kk;
        prow[kk] = j < n ? A[c * ld + j] : 0.0f;
    }
    for (int r = c + 1 + warp; r < n; r += LUM_WARPS) {
        const float l = A[r * ld + c] * inv;
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) {
            const int j = c + 1 + lane + 32 * kk;
            if (j < n) A[r * ld + j] = fmaf(-l, prow[kk], A[r * ld + j]);
        }
        __syncwarp();   // every lane has read A[r][c] before it becomes the multiplier
        if (lane == 0) A[r * ld + c] = l;
    }
}

__global__ void __launch_bounds__(LUM_THREADS, 2) lu_mixed_kernel(int n, int64_t ns, const double *__restrict__ Ag,
                                                                  const double *__restrict__ bg,
                                                                  const int32_t *__restrict__ active,
                                                                  double *__restrict__ xg,
                                                                  int32_t *__restrict__ status, double rtol) {
    extern __shared__ float4 lum_raw[];
    const int ld = n | 1;   // odd row stride: column reads hit distinct banks
    float *A = reinterpret_cast<float *>(lum_raw);
    double *x = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(lum_raw) +
                                           (((size_t)n * ld * sizeof(float) + 15) & ~(size_t)15));
    double *res = x + n;
    float *y = reinterpret_cast<float *>(res + n);
    int *perm = reinterpret_cast<int *>(y + n);
    __shared__ float pmax[LUM_WARPS];
    __shared__ int pidx[LUM_WARPS];
    __shared__ double red[LUM_WARPS];
    const int64_t s = blockIdx.x;
    if (active && !active[s]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *As = Ag + s * (int64_t)n * n;
    for (int e = tid; e < n * n; e += LUM_THREADS) {
        const int r = e / n;
        A[r * ld + (e - r * n)] = (float)As[e];
    }
    for (int r = tid; r < n; r += LUM_THREADS) perm[r] = r;
    __syncthreads();
    // factor P A = L U (rows swapped whole, as in LAPACK getrf)
    bool singular = false;
    for (int c = 0; c < n; ++c) {
        // pivot: largest |A[r][c]|, r >= c (ties: smallest r; NaN never wins)
        float best = -1.0f;
        int bi = n;
        for (int r = c + tid; r < n; r += LUM_THREADS) {
            const float a = fabsf(A[r * ld + c]);
            if (a > best) { best = a; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (b2 > best || (b2 == best && i2 < bi)) { best = b2; bi = i2; }
        }
        if (lane == 0) { pmax[warp] = best; pidx[warp] = bi; }
        __syncthreads();
        best = pmax[0];
        bi = pidx[0];
        for (int w = 1; w < LUM_WARPS; ++w)
            if (pmax[w] > best || (pmax[w] == best && pidx[w] < bi)) { best = pmax[w]; bi = pidx[w]; }
        if (!(best > 0.0f) || bi >= n) { singular = true; break; }
        if (bi != c) {
            for (int j = tid; j < n; j += LUM_THREADS) {
                const float t = A[c * ld + j];
                A[c * ld + j] = A[bi * ld + j];
                A[bi * ld + j] = t;
            }
            if (tid == 0) {
                const int t = perm[c];
                perm[c] = perm[bi];
                perm[bi] = t;
            }
        }
        __syncthreads();
        const float inv = 1.0f / A[c * ld + c];
        // the update of rows c + 1 .. n - 1, compiled for the number of 32-column
        // chunks left of the pivot row (the instruction stream is the limit; n <= 192)
        switch ((n - c + 30) >> 5) {
            case 1: lum_update_rows<1>(A, ld, n, c, inv, lane, warp); break;
            case 2: lum_update_rows<2>(A, ld, n, c, inv, lane, warp); break;
            case 3: lum_update_rows<3>(A, ld, n, c, inv, lane, warp); break;
            case 4: lum_update_rows<4>(A, ld, n, c, inv, lane, warp); break;
            case 5: lum_update_rows<5>(A, ld, n, c, inv, lane, warp); break;
            case 6: lum_update_rows<6>(A, ld, n, c, inv, lane, warp); break;
            default: break;   // c = n - 1: no rows below
        }
        __syncthreads();
    }
    if (singular) {
        if (tid == 0) status[s] = 2;
        return;
    }
    // the system A x = -r: start from x = 0, residual = -r
    for (int i = tid; i < n; i += LUM_THREADS) {
        x[i] = 0.0;
        res[i] = -bg[s * n + i];
    }
    __syncthreads();
    bool done = false;
    double dprev = HUGE_VAL;
    for (int it = 0; it < LUM_SOLVES && !done; ++it) {
        // correction d = A^-1 res through the FP32 factors (res scaled to O(1))
        // (a non-finite entry counts as infinite: fmax alone would skip a NaN)
        double sc = 0.0;
        for (int i = tid; i < n; i += LUM_THREADS) sc = fmax(sc, isfinite(res[i]) ? fabs(res[i]) : HUGE_VAL);
        sc = lum_block_max(sc, red);
        if (sc == 0.0) { done = true; break; }    // exact
        if (!(sc < HUGE_VAL)) break;              // non-finite: left to the FP64 kernel
        for (int i = tid; i < n; i += LUM_THREADS) y[i] = (float)(res[perm[i]] / sc);
        __syncthreads();
        lum_solve(A, ld, n, y);
        double dmax = 0.0, xmax = 0.0;
        for (int i = tid; i < n; i += LUM_THREADS) {
            const double d = sc * (double)y[i];
            x[i] += d;
            dmax = fmax(dmax, isfinite(d) ? fabs(d) : HUGE_VAL);
            xmax = fmax(xmax, isfinite(x[i]) ? fabs(x[i]) : HUGE_VAL);
        }
        dmax = lum_block_max(dmax, red);
        xmax = lum_block_max(xmax, red);
        if (!(xmax < HUGE_VAL)) break;
        if (dmax <= xmax * rtol) { done = true; break; }
        if (it > 0 && !(dmax <= 0.5 * dprev)) break;   // not converging: left to FP64
        dprev = dmax;
        // residual -r - A x in FP64 (a warp per row, lanes along the row)
        for (int r = warp; r < n; r += LUM_WARPS) {
            double acc = 0.0;
            for (int j = lane; j < n; j += 32) acc = fma(As[(int64_t)r * n + j], x[j], acc);
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) res[r] = -bg[s * n + r] - acc;
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += LUM_THREADS) xg[s * n + i] = x[i];
    if (tid == 0) status[s] = done ? 0 : 3;
}

// ---------------------------------------------------------------------------
// Newton helpers: norms, trial points, acceptance
// ---------------------------------------------------------------------------

__global__ void norms_kernel(int n, int64_t ns, const double *__restrict__ r, double *__restrict__ n2,
                             double *__restrict__ ninf) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    double a = 0.0, b = 0.0;
    for (int j = 0; j < n; ++j) {
        const double v = r[s * n + j];
        a += v * v;
        b = fmax(b, fabs(v));
        if (!isfinite(v)) { a = INFINITY; b = INFINITY; }
    }
    n2[s] = sqrt(a);
    ninf[s] = b;
}

// z[s] = zt[s] for the states whose trial point was accepted
__global__ void accept_kernel(int n, int64_t ns, const int32_t *__restrict__ acc, const double *__restrict__ zt,
                              double *__restrict__ z) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ns * n) return;
    if (acc[e / n]) z[e] = zt[e];
}

// dst row k = src row kidx[k] (rows of w doubles): the Newton working set compacted
__global__ void gather_rows_kernel(int64_t nk, int w, const int32_t *__restrict__ kidx, const double *__restrict__ src,
                                   double *__restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nk * w) return;
    const int64_t k = e / w;
    dst[e] = src[(int64_t)kidx[k] * w + (e - k * w)];
}

// dst row widx[k] = src row k: the working set's solutions back to the caller's array
__global__ void scatter_rows_kernel(int64_t nk, int w, const int64_t *__restrict__ widx, const double *__restrict__ src,
                                    double *__restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nk * w) return;
    const int64_t k = e / w;
    dst[widx[k] * w + (e - k * w)] = src[e];
}

__global__ void trial_kernel(int n, int64_t ns, const double *__restrict__ z, const double *__restrict__ dz,
                             const double *__restrict__ step, const int32_t *__restrict__ active,
                             double *__restrict__ zt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ns * n) return;
    const int64_t s = e / n;
    zt[e] = active[s] ? z[e] + step[s] * dz[e] : z[e];
}

// ---------------------------------------------------------------------------
// node shortcut: the 2(N+1) next states of one state differ only in a'. For a
// country node (2i or 2i+1) only a'_i moves off its no-shock value, so the
// policy there is the no-shock policy plus, for each component holding a_i,
// that component at the shocked a'_i minus it at the no-shock a'_i. Only the
// no-shock state and the two global-shock nodes (2N, 2N+1: every a' shocked)
// are interpolated in full.
// ---------------------------------------------------------------------------

// 3 queries per state: 0 no shock, 1 every country +, 2 every country - (the
// global nodes). Clamps are counted with the multiplicity the 2(N+1) node
// queries would have, so the clamp counter agrees with the full path.
__global__ void irbc_queries3_kernel(IrbcDev P, int64_t ns, const double *__restrict__ states,
                                     const double *__restrict__ guess, const double *__restrict__ lo,
                                     const double *__restrict__ span, uint64_t *__restrict__ X,
                                     int32_t *__restrict__ flags, unsigned long long *__restrict__ stats) {
    const int N = P.N, d = 2 * N, m = P.m, nq = 2 * (N + 1);
    const int64_t Q3 = ns * 3;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long clamps = 0;
    if (idx < ns * d) {
        const int64_t s = idx / d;
        const int dim = (int)(idx - s * d);
        bool bad = false;
        uint64_t *Xrow = X + (int64_t)dim * Q3 + s * 3;
        if (dim < N) {
            double v[3];
            next_a3(P, states[s * d + dim], v[0], v[1], v[2]);
            const unsigned long long mult[3] = {(unsigned long long)(nq - 4), 2ull, 2ull};
            for (int t = 0; t < 3; ++t) {
                unsigned long long c1 = 0;
                Xrow[t] = encode_coord(v[t], lo[dim], span[dim], bad, c1);
                clamps += c1 * mult[t];
            }
            if (!isfinite(states[s * d + N + dim])) bad = true;
        } else {
            const uint64_t e = encode_coord(guess[s * m + dim - N], lo[dim], span[dim], bad, clamps);
            clamps *= (unsigned long long)nq;
            for (int t = 0; t < 3; ++t) Xrow[t] = e;
            if (dim == d - 1)
                for (int o = N; o < m; ++o)
                    if (!isfinite(guess[s * m + o])) bad = true;
        }
        if (bad)
            for (int t = 0; t < 3; ++t) flags[s * 3 + t] = 1;
    }
    for (int o = 16; o > 0; o >>= 1) clamps += __shfl_down_sync(0xffffffffu, clamps, o);
    if ((threadIdx.x & 31) == 0 && clamps) atomicAdd(&stats[0], clamps);
}

// Node shortcut (one thread per (state, country i) for the term search, then
// one warp per 32 such pairs for the sums). The policy at the two nodes that
// shock country i (2i: +, 2i+1: -) is the no-shock policy plus the change of
// every component holding a_i when a'_i moves to its shocked value. Writes
// those changes, dY (2N rows of m per state, in W), which the residual and
// Jacobian kernels read beside the no-shock and global-shock rows.
// Phase 1: each thread encodes a'_i's three values (no shock, +, -) and walks
// the tuples of its components once, keeping the active (row, weight) term of
// every value in shared memory (at most DLT_CAP per value; a pair with more
// is flagged). Phase 2: the warp takes its 32 pairs in turn, lanes over the
// outputs (o, o + 32, ...), and sums weight x surplus row over each value's
// terms in (component, tuple) order, DLT_UNR terms' rows in flight at a time;
// every surplus row is read and every policy row written coalesced. A
// flagged pair is summed by a warp-wide walk of its tuples (lanes over the
// tuples, active terms broadcast in the same order). Changes = sum_v - sum_0,
// the sums and their difference in W (no FP64 arithmetic per output).
constexpr int DLT_WARPS = 4;   // warps per block
constexpr int DLT_CAP = 16;    // terms per (pair, value) kept in shared memory

template <class W>
struct DltTerms {   // one warp's term lists, lane (pair) fastest
    int32_t row[3][DLT_CAP][32];
    W w[3][DLT_CAP][32];
};

template <int PREC>
constexpr int dlt_unroll() { return PREC == DDSG_F64 ? 2 : 4; }

// Coordinates of component cd at state s with a'_i in Xd[ipos] = Xi0 (the
// other a-dimensions at their no-shock values, k-dimensions at the guess).
__device__ __forceinline__ int delta_coords(const IrbcDev &P, const DevComp &cd, int i, int64_t s,
                                            const double *states, const double *guess, const double *lo,
                                            const double *span, uint64_t Xi0, uint64_t *Xd, bool &bad) {
    const int N = P.N, d = 2 * N, m = P.m;
    unsigned long long cl = 0;
    int ipos = 0;
    for (int j = 0; j < cd.k; ++j) {
        const int dj = cd.dims[j];
        if (dj == i) {
            ipos = j;
            Xd[j] = Xi0;
        } else if (dj < N) {
            double f0, fp, fm;
            next_a3(P, states[s * d + dj], f0, fp, fm);
            Xd[j] = encode_coord(f0, lo[dj], span[dj], bad, cl);
        } else {
            Xd[j] = encode_coord(guess[s * m + dj - N], lo[dj], span[dj], bad, cl);
        }
    }
    return ipos;
}

// (row, weight) of tuple tu at coordinates Xd; row -1 when inactive. The
// weight is coef times the hat values, in W (the hat values built from their
// fixed-point bits as in the evaluation kernels: no FP64 work for W = float).
template <class W>
__device__ __forceinline__ int32_t delta_term(const DevTables &t, const DevComp &cd, const DevTup &tu,
                                              const uint64_t *Xd, W coef, W &w) {
    uint32_t off = 0;
    w = coef;
    for (int j = 0; j < cd.k; ++j) {
        Basis1D o;
        const int l = tu.lev[j];
        if (!basis1d(Xd[j], l, o)) return -1;
        off = off * (j == 1 ? tu.nc1 : ncells(l)) + o.cell;
        w *= basis_val<W>(o);
    }
    return tuple_row_at(tu, off, t.slots, t.S, cd.row_begin, cd.row_end);
}

// Warp-wide walk for one pair whose terms did not fit: acc[v][c] += the sum for
// value v at outputs m0 + lane + 32c. Returns false on a non-finite coordinate.
template <int PREC, int OC>
__device__ __forceinline__ bool delta_walk_warp(const IrbcDev &P, const DevTables &t, bool paper, const int32_t *aoff,
                                const int32_t *acomp, const double *states, const double *guess,
                                const double *lo, const double *span, int64_t s, int i, const uint64_t (&Xi)[3],
                                int m0, int lane, typename DeltaT<PREC>::W (&acc)[3][OC]) {
    using W = typename DeltaT<PREC>::W;
    const W *alpha = DeltaT<PREC>::alpha(t);
    const int mp = DeltaT<PREC>::stride(t);
    const int m = P.m, d = 2 * P.N;
    for (int e = aoff[i]; e < aoff[i + 1]; ++e) {
        if (!comp_ok(t, acomp[e], d)) continue;
        const DevComp &cd = t.comps[acomp[e]];
        const double coef = paper ? cd.b : 1.0;
        if (coef == 0.0) continue;
        uint64_t Xd[KMAX];
        bool bad = false;
        const int ipos = delta_coords(P, cd, i, s, states, guess, lo, span, Xi[0], Xd, bad);
        if (bad) return false;
        const int tb = paper ? cd.tup_begin : cd.tup_int;
        for (int t0 = tb; t0 < cd.tup_end; t0 += 32) {
            const int ti = t0 + lane;
            int32_t row[3] = {-1, -1, -1};
            W wv[3] = {(W)0, (W)0, (W)0};
            if (ti < cd.tup_end) {
                const DevTup tu = t.tups[ti];
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    Xd[ipos] = Xi[v];
                    row[v] = delta_term<W>(t, cd, tu, Xd, (W)coef, wv[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                unsigned mask = __ballot_sync(0xffffffffu, row[v] >= 0);
                while (mask) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int32_t r = __shfl_sync(0xffffffffu, row[v], src);
                    const W ww = __shfl_sync(0xffffffffu, wv[v], src);
                    const W *a = alpha + (int64_t)r * mp;
#pragma unroll
                    for (int c = 0; c < OC; ++c) {
                        const int o = m0 + lane + 32 * c;
                        if (o < m) acc[v][c] += ww * a[o];
                    }
                }
            }
        }
    }
    return true;
}

template <int PREC, int OC>
__global__ void __launch_bounds__(32 * DLT_WARPS) irbc_delta_kernel(IrbcDev P, int64_t s0, int64_t nsc, DevTables t,
                                                                    int form, const int32_t *__restrict__ aoff,
                                                                    const int32_t *__restrict__ acomp,
                                                                    const double *__restrict__ states,
                                                                    const double *__restrict__ guess,
                                                                    const double *__restrict__ lo,
                                                                    const double *__restrict__ span,
                                                                    const double *__restrict__ y3,
                                                                    typename DeltaT<PREC>::W *__restrict__ dY) {
    using W = typename DeltaT<PREC>::W;
    constexpr int UNR = dlt_unroll<PREC>();
    const W *alpha = DeltaT<PREC>::alpha(t);
    const int mp = DeltaT<PREC>::stride(t);
    const int N = P.N, d = 2 * N, m = P.m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool paper = form == DDSG_FORM_PAPER;
    extern __shared__ float4 dlt_raw[];
    DltTerms<W> &T = reinterpret_cast<DltTerms<W> *>(dlt_raw)[warp];
    const int64_t npairs = nsc * N;
    const int64_t wbase = ((int64_t)blockIdx.x * DLT_WARPS + warp) * 32;
    if (wbase >= npairs) return;   // whole warps leave together
    // phase 1: this lane's pair
    const int64_t pair = wbase + lane;
    int64_t sl = 0;
    int i = 0;
    bool bad = false, over = false;
    int cnt[3] = {0, 0, 0};
    uint64_t Xi[3] = {0, 0, 0};
    if (pair < npairs) {
        sl = pair / N;
        i = (int)(pair - sl * N);
        const int64_t s = s0 + sl;
        unsigned long long cl = 0;
        double e3[3];
        next_a3(P, states[s * d + i], e3[0], e3[1], e3[2]);
        for (int v = 0; v < 3; ++v) Xi[v] = encode_coord(e3[v], lo[i], span[i], bad, cl);
        for (int e = aoff[i]; e < aoff[i + 1] && !bad && !over; ++e) {
            if (!comp_ok(t, acomp[e], d)) continue;
            const DevComp &cd = t.comps[acomp[e]];
            const double coef = paper ? cd.b : 1.0;
            if (coef == 0.0) continue;
            uint64_t Xd[KMAX];
            const int ipos = delta_coords(P, cd, i, s, states, guess, lo, span, Xi[0], Xd, bad);
            if (bad) break;
            const int tb = paper ? cd.tup_begin : cd.tup_int;
            for (int ti = tb; ti < cd.tup_end && !over; ++ti) {
                const DevTup tu = t.tups[ti];
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    Xd[ipos] = Xi[v];
                    W w;
                    const int32_t r = delta_term<W>(t, cd, tu, Xd, (W)coef, w);
                    if (r < 0) continue;
                    if (cnt[v] == DLT_CAP) { over = true; break; }
                    T.row[v][cnt[v]][lane] = r;
                    T.w[v][cnt[v]][lane] = w;
                    ++cnt[v];
                }
            }
        }
    }
    __syncwarp();
    // phase 2: the warp's pairs in turn
    const int np = npairs - wbase < 32 ? (int)(npairs - wbase) : 32;
    for (int p = 0; p < np; ++p) {
        const int64_t slp = __shfl_sync(0xffffffffu, sl, p);
        const int ip = __shfl_sync(0xffffffffu, i, p);
        const bool badp = __shfl_sync(0xffffffffu, (int)bad, p) != 0;
        const bool overp = __shfl_sync(0xffffffffu, (int)over, p) != 0;
        int cp[3];
        uint64_t Xp[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            cp[v] = __shfl_sync(0xffffffffu, cnt[v], p);
            Xp[v] = __shfl_sync(0xffffffffu, Xi[v], p);
        }
        W *dp_row = dY + (slp * 2 * N + 2 * ip) * (int64_t)m;   // node 2i (+); node 2i + 1 (-) follows
        W *dm_row = dp_row + m;
        for (int m0 = 0; m0 < m; m0 += 32 * OC) {
            W acc[3][OC];
#pragma unroll
            for (int v = 0; v < 3; ++v)
#pragma unroll
                for (int c = 0; c < OC; ++c) acc[v][c] = (W)0;
            bool nan = badp;
            if (!badp && overp) {
                nan = !delta_walk_warp<PREC, OC>(P, t, paper, aoff, acomp, states, guess, lo, span, s0 + slp, ip, Xp,
                                                 m0, lane, acc);
            } else if (!badp) {
                bool ok[OC];   // this lane's outputs in range
#pragma unroll
                for (int c = 0; c < OC; ++c) ok[c] = m0 + lane + 32 * c < m;
                const W *al = alpha + m0 + lane;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int n = cp[v];
                    int q = 0;
                    for (; q + UNR <= n; q += UNR) {   // UNR terms' rows in flight
                        int32_t r[UNR];
                        W ww[UNR], x[UNR][OC];
#pragma unroll
                        for (int k = 0; k < UNR; ++k) {
                            r[k] = T.row[v][q + k][p];
                            ww[k] = T.w[v][q + k][p];
                        }
#pragma unroll
                        for (int k = 0; k < UNR; ++k)
#pragma unroll
                            for (int c = 0; c < OC; ++c) x[k][c] = ok[c] ? al[(int64_t)r[k] * mp + 32 * c] : (W)0;
#pragma unroll
                        for (int k = 0; k < UNR; ++k)
#pragma unroll
                            for (int c = 0; c < OC; ++c) acc[v][c] += ww[k] * x[k][c];
                    }
                    for (; q < n; ++q) {   // the rest, one term at a time (same order)
                        const int32_t r = T.row[v][q][p];
                        const W ww = T.w[v][q][p];
#pragma unroll
                        for (int c = 0; c < OC; ++c)
                            if (ok[c]) acc[v][c] += ww * al[(int64_t)r * mp + 32 * c];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < OC; ++c) {
                const int o = m0 + lane + 32 * c;
                if (o < m) {
                    dp_row[o] = nan ? (W)NAN : acc[1][c] - acc[0][c];
                    dm_row[o] = nan ? (W)NAN : acc[2][c] - acc[0][c];
                }
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct irbc {
    irbc_params_t p;
    int node_mode = DDSG_IRBC_NODES_ALL;
    int irreversible = 0;   // non-smooth model: policy (k', mu, lambda)
    Tracer tr;   // kinds: 0 queries, 1 eval, 2 residual, 3 jacobian, 4 lu, 5 newton helpers
    std::vector<double> gamma, tau;
    int device = -1;
    double *gamma_d = nullptr, *tau_d = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *nws = nullptr;      // Newton buffers (kept between solves)
    size_t nws_bytes = 0;
};

namespace {

int ensure(irbc *M, size_t bytes) {
    if (bytes <= M->ws_bytes) return DDSG_OK;
    cudaFree(M->ws);
    M->ws = nullptr;
    M->ws_bytes = 0;
    if (dev_alloc(&M->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DDSG_ERR_OOM, "IRBC workspace allocation failed");
    }
    M->ws_bytes = bytes;
    return DDSG_OK;
}

IrbcDev dev_params(const irbc *M) {
    IrbcDev P;
    P.N = M->p.N;
    P.irr = M->irreversible;
    P.m = M->irreversible ? 2 * M->p.N + 1 : M->p.N + 1;
    P.beta = M->p.beta;
    P.alpha = M->p.alpha;
    P.delta = M->p.delta;
    P.sigma = M->p.sigma;
    P.rho = M->p.rho;
    P.phi = M->p.phi;
    P.A = M->p.A;
    P.shk_p = std::exp(M->p.sigma * std::sqrt((double)(M->p.N + 1)));
    P.shk_m = std::exp(-M->p.sigma * std::sqrt((double)(M->p.N + 1)));
    P.gamma = M->gamma_d;
    P.tau = M->tau_d;
    return P;
}

constexpr size_t kWsCap = (size_t)2 << 30;   // residual workspace per chunk of states

// CSR over the dims N+i (the k_i): the components that hold k_i. Fails if one
// of them also holds more than one a-dimension (the Jacobian kernel handles
// at most one shocked coordinate per component).
// terms: the most derivative terms one state's Jacobian can collect in `form`
// (each level tuple gives at most one per a'-value of its component, and the
// kernel keeps at most DT_CAP per group and value).
int k_components(hdmr_t *h, int N, int form, std::vector<int32_t> &off, std::vector<int32_t> &ids,
                 int64_t &terms) {
    int32_t nc = 0;
    int64_t np = 0;
    int rc = hdmr_num_components(h, &nc, &np);
    if (rc) return rc;
    std::vector<int32_t> ntup;
    if ((rc = handle_comp_tuples(h, form, ntup))) return rc;
    std::vector<std::vector<int32_t>> per(N);
    terms = 0;
    for (int32_t c = 0; c < nc; ++c) {
        int32_t kk = 0, dims[DDSG_KMAX];
        hdmr_component_info(h, c, &kk, dims, nullptr, nullptr);
        int na = 0;
        for (int j = 0; j < kk; ++j) na += dims[j] < N;
        for (int j = 0; j < kk; ++j) {
            if (dims[j] < N) continue;
            if (na > 1)
                return set_error(DDSG_ERR_ARG, "euler_residual: the Jacobian needs every component holding a k_i to hold at most one a_j");
            per[dims[j] - N].push_back(c);
            terms += (int64_t)(na ? 3 : 1) * std::min<int32_t>(ntup[c], DT_CAP);
        }
    }
    off.assign(N + 1, 0);
    ids.clear();
    for (int i = 0; i < N; ++i) {
        ids.insert(ids.end(), per[i].begin(), per[i].end());
        off[i + 1] = (int32_t)ids.size();
    }
    return DDSG_OK;
}

// CSR over the dims i < N (the a_i): the components that hold a_i.
int a_components(hdmr_t *h, int N, std::vector<int32_t> &off, std::vector<int32_t> &ids) {
    int32_t nc = 0;
    int64_t np = 0;
    int rc = hdmr_num_components(h, &nc, &np);
    if (rc) return rc;
    std::vector<std::vector<int32_t>> per(N);
    for (int32_t c = 0; c < nc; ++c) {
        int32_t kk = 0, dims[DDSG_KMAX];
        hdmr_component_info(h, c, &kk, dims, nullptr, nullptr);
        for (int j = 0; j < kk; ++j)
            if (dims[j] < N) per[dims[j]].push_back(c);
    }
    off.assign(N + 1, 0);
    ids.clear();
    for (int i = 0; i < N; ++i) {
        ids.insert(ids.end(), per[i].begin(), per[i].end());
        off[i + 1] = (int32_t)ids.size();
    }
    return DDSG_OK;
}

template <int PREC, int OC>
cudaError_t launch_delta_oc(const IrbcDev &P, int64_t s0, int64_t nsc, const DevTables &t, int form,
                            const int32_t *aoff, const int32_t *acomp, const double *states, const double *guess,
                            const double *lo, const double *span, const double *y3,
                            typename DeltaT<PREC>::W *dY, cudaStream_t st) {
    const size_t smem = sizeof(DltTerms<typename DeltaT<PREC>::W>) * DLT_WARPS;
    cudaError_t e = cudaFuncSetAttribute(irbc_delta_kernel<PREC, OC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t warps = (nsc * P.N + 31) / 32;
    irbc_delta_kernel<PREC, OC><<<(unsigned)((warps + DLT_WARPS - 1) / DLT_WARPS), 32 * DLT_WARPS, smem, st>>>(
        P, s0, nsc, t, form, aoff, acomp, states, guess, lo, span, y3, dY);
    return cudaGetLastError();
}

// outputs per lane per pass: the fewest of 2, 4, 5, 6, 8 that cover m in one pass
template <int PREC>
cudaError_t launch_delta(const IrbcDev &P, int64_t s0, int64_t nsc, const DevTables &t, int form,
                         const int32_t *aoff, const int32_t *acomp, const double *states, const double *guess,
                         const double *lo, const double *span, const double *y3, typename DeltaT<PREC>::W *dY,
                         cudaStream_t st) {
    const int need = (P.m + 31) / 32;
    if (need <= 2) return launch_delta_oc<PREC, 2>(P, s0, nsc, t, form, aoff, acomp, states, guess, lo, span, y3, dY, st);
    if (need <= 4) return launch_delta_oc<PREC, 4>(P, s0, nsc, t, form, aoff, acomp, states, guess, lo, span, y3, dY, st);
    if (need <= 5) return launch_delta_oc<PREC, 5>(P, s0, nsc, t, form, aoff, acomp, states, guess, lo, span, y3, dY, st);
    if (need <= 6) return launch_delta_oc<PREC, 6>(P, s0, nsc, t, form, aoff, acomp, states, guess, lo, span, y3, dY, st);
    return launch_delta_oc<PREC, 8>(P, s0, nsc, t, form, aoff, acomp, states, guess, lo, span, y3, dY, st);
}

}  // namespace

extern "C" int irbc_set_irreversible(irbc_t *M, int on) {
    if (!M) return set_error(DDSG_ERR_ARG, "irbc_set_irreversible: NULL model");
    if (on && 2 * M->p.N + 1 > 165)
        return set_error(DDSG_ERR_ARG, "irbc_set_irreversible: 2N+1 > 165 unknowns per state (batched LU limit)");
    M->irreversible = on ? 1 : 0;
    return DDSG_OK;
}

extern "C" int irbc_set_node_mode(irbc_t *M, int mode) {
    if (!M) return set_error(DDSG_ERR_ARG, "irbc_set_node_mode: NULL model");
    if (mode != DDSG_IRBC_NODES_ALL && mode != DDSG_IRBC_NODES_DELTA)
        return set_error(DDSG_ERR_ARG, "irbc_set_node_mode: unknown mode");
    M->node_mode = mode;
    return DDSG_OK;
}

extern "C" int irbc_create(const irbc_params_t *prm, const double *gamma_host, const double *tau_host,
                           irbc_t **out) {
    if (!prm || !gamma_host || !tau_host || !out) return set_error(DDSG_ERR_ARG, "irbc_create: NULL argument");
    if (prm->N < 1 || prm->N > 4096) return set_error(DDSG_ERR_ARG, "irbc_create: N out of range");
    irbc *M = new (std::nothrow) irbc();
    if (!M) return set_error(DDSG_ERR_OOM, "irbc_create: host allocation failed");
    M->p = *prm;
    M->gamma.assign(gamma_host, gamma_host + prm->N);
    M->tau.assign(tau_host, tau_host + prm->N);
    *out = M;
    return DDSG_OK;
}

// Table 1 of the paper: productivity A = (1 - beta (1 - delta)) / (alpha beta),
// utility curvatures gamma_j = a + 0.75 (j - 1) / (N - 1) (a alone when N = 1,
// j = 1..N) and weights tau_j = A^(1 / gamma_j), so that the steady state has
// k_j = 1 for every country.
extern "C" int irbc_create_table1(int N, double a_gamma, double beta, double alpha, double delta, double sigma,
                                  double rho, double phi, irbc_t **out) {
    if (!out) return set_error(DDSG_ERR_ARG, "irbc_create_table1: NULL argument");
    if (N < 1 || N > 4096) return set_error(DDSG_ERR_ARG, "irbc_create_table1: N out of range");
    if (!(beta > 0.0 && beta < 1.0) || !(alpha > 0.0 && alpha < 1.0) || !(delta >= 0.0 && delta < 1.0) ||
        !(a_gamma > 0.0))
        return set_error(DDSG_ERR_ARG, "irbc_create_table1: parameter out of range");
    irbc_params_t prm;
    prm.N = N;
    prm.beta = beta;
    prm.alpha = alpha;
    prm.delta = delta;
    prm.sigma = sigma;
    prm.rho = rho;
    prm.phi = phi;
    prm.A = (1.0 - beta * (1.0 - delta)) / (alpha * beta);
    std::vector<double> gamma(N), tau(N);
    for (int j = 0; j < N; ++j) {
        gamma[j] = N > 1 ? a_gamma + 0.75 * (double)j / (double)(N - 1) : a_gamma;
        tau[j] = pow(prm.A, 1.0 / gamma[j]);
    }
    return irbc_create(&prm, gamma.data(), tau.data(), out);
}

extern "C" int irbc_get_params(const irbc_t *M, irbc_params_t *prm, double *gamma_host, double *tau_host) {
    if (!M) return set_error(DDSG_ERR_ARG, "irbc_get_params: NULL model");
    if (prm) *prm = M->p;
    if (gamma_host) std::copy(M->gamma.begin(), M->gamma.end(), gamma_host);
    if (tau_host) std::copy(M->tau.begin(), M->tau.end(), tau_host);
    return DDSG_OK;
}

extern "C" int irbc_destroy(irbc_t *M) {
    if (!M) return DDSG_OK;
    cudaFree(M->gamma_d);
    cudaFree(M->tau_d);
    cudaFree(M->ws);
    cudaFree(M->nws);
    delete M;
    return DDSG_OK;
}

static int bind_device(irbc *M) {
    if (M->device >= 0) return DDSG_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(DDSG_ERR_CUDA, "IRBC: no CUDA device");
    const size_t nb = sizeof(double) * M->p.N;
    if (dev_alloc(&M->gamma_d, nb) != cudaSuccess || dev_alloc(&M->tau_d, nb) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(M->gamma_d);
        cudaFree(M->tau_d);
        M->gamma_d = M->tau_d = nullptr;
        return set_error(DDSG_ERR_OOM, "IRBC: parameter buffers unavailable");
    }
    if (cudaMemcpy(M->gamma_d, M->gamma.data(), nb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(M->tau_d, M->tau.data(), nb, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DDSG_ERR_CUDA, "IRBC: parameter upload failed");
    }
    M->device = dev;
    return DDSG_OK;
}

extern "C" int euler_residual(irbc_t *M, hdmr_t *policy, int64_t ns, const double *states_dev,
                              const double *guess_dev, double *resid_dev, double *jac_dev,
                              double *euler_err_dev, int precision, int form, ddsg_stream_t stream) {
    if (!M || !policy || ns < 0 || (ns > 0 && (!states_dev || !guess_dev || !resid_dev)))
        return set_error(DDSG_ERR_ARG, "euler_residual: bad argument");
    if (ns == 0) return DDSG_OK;
    HandleView v;
    int rc = handle_eval_view(policy, precision, form, &v);
    if (rc) return rc;
    const int N = M->p.N, d = 2 * N, m = M->irreversible ? 2 * N + 1 : N + 1, nq = 2 * (N + 1);
    if (v.d != d || v.m != m)
        return set_error(DDSG_ERR_ARG, M->irreversible ? "euler_residual: the policy must map 2N states to 2N+1 outputs (k', mu, lambda)"
                                                       : "euler_residual: the policy must map 2N states to N+1 outputs");
    if ((rc = bind_device(M))) return rc;
    std::vector<int32_t> koff, kids;
    int64_t jac_terms = 0;
    int32_t *koff_dev = nullptr, *kids_dev = nullptr;
    if (jac_dev) {
        if ((rc = k_components(policy, N, form, koff, kids, jac_terms))) return rc;
        if (N > 32 * JAC_KJ)
            return set_error(DDSG_ERR_ARG, "euler_residual: the Jacobian supports N <= 192");
        if (((sizeof(JGroup) * kids.size() + sizeof(int32_t) * N + 15) & ~(size_t)15) +
                ((sizeof(double) * 12 * N + 15) & ~(size_t)15) + sizeof(uint64_t) * 4 * N +
                64 * sizeof(DTerm<double>) > kJacSmem)
            return set_error(DDSG_ERR_ARG, "euler_residual: too many components hold a k dimension for the Jacobian");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool delta = M->node_mode == DDSG_IRBC_NODES_DELTA;
    std::vector<int32_t> aoff, acomp;
    if (delta && (rc = a_components(policy, N, aoff, acomp))) return rc;
    // interpolated queries per state: all 2(N+1) nodes, or (node shortcut) the
    // no-shock state and the two global-shock nodes
    const int nqe = delta ? 3 : nq;
    // per state: X (d*nqe*8) + flags (nqe*4) + y of the shortcut's 3 queries + y
    // of all nodes (nq*m*8) + aux (7N*8)
    const size_t per_state = (size_t)nqe * (d * 8 + 4) + (delta ? (size_t)3 * m * 8 : 0) +
                             (size_t)nq * m * 8 + (size_t)7 * N * 8;
    int64_t chunk = std::max<int64_t>(1, (int64_t)(kWsCap / per_state));
    chunk = std::min<int64_t>(chunk, ns);
    auto rnd = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t kc_bytes = jac_dev ? rnd(sizeof(int32_t) * koff.size()) + rnd(sizeof(int32_t) * (kids.size() + 1)) : 0;
    const size_t ac_bytes = delta ? rnd(sizeof(int32_t) * aoff.size()) + rnd(sizeof(int32_t) * (acomp.size() + 1)) : 0;
    if ((rc = ensure(M, per_state * chunk + 4096 + kc_bytes + ac_bytes))) return rc;
    unsigned char *base = static_cast<unsigned char *>(M->ws);
    if (jac_dev) {
        koff_dev = reinterpret_cast<int32_t *>(base);
        kids_dev = reinterpret_cast<int32_t *>(base + rnd(sizeof(int32_t) * koff.size()));
        if (cudaMemcpyAsync(koff_dev, koff.data(), sizeof(int32_t) * koff.size(), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            (!kids.empty() && cudaMemcpyAsync(kids_dev, kids.data(), sizeof(int32_t) * kids.size(),
                                              cudaMemcpyHostToDevice, st) != cudaSuccess))
            return set_error(DDSG_ERR_CUDA, "euler_residual: copy failed");
        base += kc_bytes;
    }
    int32_t *aoff_dev = nullptr, *acomp_dev = nullptr;
    if (delta) {
        aoff_dev = reinterpret_cast<int32_t *>(base);
        acomp_dev = reinterpret_cast<int32_t *>(base + rnd(sizeof(int32_t) * aoff.size()));
        if (cudaMemcpyAsync(aoff_dev, aoff.data(), sizeof(int32_t) * aoff.size(), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            (!acomp.empty() && cudaMemcpyAsync(acomp_dev, acomp.data(), sizeof(int32_t) * acomp.size(),
                                               cudaMemcpyHostToDevice, st) != cudaSuccess))
            return set_error(DDSG_ERR_CUDA, "euler_residual: copy failed");
        base += ac_bytes;
    }
    const IrbcDev P = dev_params(M);
    for (int64_t s0 = 0; s0 < ns; s0 += chunk) {
        const int64_t nsc = std::min<int64_t>(chunk, ns - s0);
        const int64_t Q = nsc * nq, Qe = nsc * nqe;
        uint64_t *X = reinterpret_cast<uint64_t *>(base);
        int32_t *flags = reinterpret_cast<int32_t *>(X + (int64_t)d * Qe);
        double *y3 = reinterpret_cast<double *>(((uintptr_t)(flags + Qe) + 255) & ~(uintptr_t)255);
        double *y = delta ? y3 + Qe * m : y3;   // shortcut: the country nodes' changes dY, in W
        double *aux = y + Q * m;
        cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int32_t) * Qe, st);
        if (e == cudaSuccess) {
            Tracer::Scope ts(&M->tr, 0, st);
            const int64_t th = nsc * d;
            if (delta)
                irbc_queries3_kernel<<<(unsigned)((th + 255) / 256), 256, 0, st>>>(
                    P, nsc, states_dev + s0 * d, guess_dev + s0 * m, v.lo, v.span, X, flags,
                    reinterpret_cast<unsigned long long *>(v.stats));
            else
                irbc_queries_kernel<<<(unsigned)((th + 255) / 256), 256, 0, st>>>(
                    P, nsc, states_dev + s0 * d, guess_dev + s0 * m, v.lo, v.span, X, flags,
                    reinterpret_cast<unsigned long long *>(v.stats));
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            EvalArgs a;
            a.t = v.tables;
            a.d = d;
            a.m = m;
            a.n = Qe;
            a.X = X;
            a.y = y3;
            a.hash = nullptr;
            a.count = nullptr;
            a.form = form;
            a.precision = precision;
            a.cfg = v.cfg;
            a.err = reinterpret_cast<unsigned long long *>(v.stats + 2);
            Tracer::Scope ts(&M->tr, 1, st);
            e = launch_eval(a, st);
        }
        if (e == cudaSuccess && delta) {
            Tracer::Scope ts(&M->tr, 6, st);
            if (precision == DDSG_F64)
                e = launch_delta<DDSG_F64>(P, s0, nsc, *v.tables, form, aoff_dev, acomp_dev, states_dev,
                                               guess_dev, v.lo, v.span, y3, y, st);
            else
                e = launch_delta<DDSG_F32C>(P, s0, nsc, *v.tables, form, aoff_dev, acomp_dev, states_dev,
                                                guess_dev, v.lo, v.span, y3, reinterpret_cast<float *>(y), st);
        }
        if (e == cudaSuccess) {
            Tracer::Scope ts(&M->tr, 2, st);
            const int rt = std::min(RES_THREADS, (N + 31) / 32 * 32);
            const unsigned nb = (unsigned)nsc;
            if (!delta)
                irbc_residual_kernel<false, double><<<nb, rt, 0, st>>>(
                    P, s0, nsc, states_dev, guess_dev, NodePolicy<false, double>{y, nullptr, nullptr}, resid_dev,
                    euler_err_dev, jac_dev, aux);
            else if (precision == DDSG_F64)
                irbc_residual_kernel<true, double><<<nb, rt, 0, st>>>(
                    P, s0, nsc, states_dev, guess_dev, NodePolicy<true, double>{nullptr, y3, y}, resid_dev,
                    euler_err_dev, jac_dev, aux);
            else
                irbc_residual_kernel<true, float><<<nb, rt, 0, st>>>(
                    P, s0, nsc, states_dev, guess_dev,
                    NodePolicy<true, float>{nullptr, y3, reinterpret_cast<const float *>(y)}, resid_dev,
                    euler_err_dev, jac_dev, aux);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && jac_dev) {
            Tracer::Scope ts(&M->tr, 3, st);
            e = launch_jacobian(precision, P, s0, nsc, *v.tables, form, (int)kids.size(), jac_terms, koff_dev,
                                kids_dev, v.lo, v.span, guess_dev, delta ? y3 : y, delta ? (const void *)y : nullptr,
                                aux, jac_dev, st);
        }
        if (e != cudaSuccess) return set_error(DDSG_ERR_CUDA, cudaGetErrorString(e));
    }
    return DDSG_OK;
}

namespace {

// dx = -A^-1 r for the systems with active[s] != 0 (all when active is null):
// FP32 factors refined in FP64 until the correction is below rtol of the
// solution, then the FP64 kernel for those it could not refine
int lu_solve_masked(int n, int64_t ns, const double *A_dev, const double *r_dev, const int32_t *active,
                    double *dx_dev, int32_t *status_dev, double rtol, cudaStream_t st) {
    const size_t smem = sizeof(double) * ((size_t)n * n + n);
    const size_t smem_m = lum_smem_bytes(n);
    cudaError_t e = cudaFuncSetAttribute(lu_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_m);
    if (e == cudaSuccess) {
        lu_mixed_kernel<<<(unsigned)ns, LUM_THREADS, smem_m, st>>>(n, ns, A_dev, r_dev, active, dx_dev, status_dev,
                                                                   rtol);
        e = cudaGetLastError();
    }
    // the systems the FP32 factors could not refine (status 3), again in FP64
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lu_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        lu_solve_kernel<<<(unsigned)ns, 256, smem, st>>>(n, ns, A_dev, r_dev, active, dx_dev, status_dev, 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(DDSG_ERR_CUDA, cudaGetErrorString(e));
    return DDSG_OK;
}

}  // namespace

extern "C" int irbc_lu_solve(int n, int64_t ns, const double *A_dev, const double *r_dev, double *dx_dev,
                             int32_t *status_dev, ddsg_stream_t stream) {
    if (n < 1 || ns < 0) return set_error(DDSG_ERR_ARG, "irbc_lu_solve: bad size");
    if (ns == 0) return DDSG_OK;
    const size_t smem = sizeof(double) * ((size_t)n * n + n);
    if (smem > 220 * 1024) return set_error(DDSG_ERR_ARG, "irbc_lu_solve: system too large for shared memory (n <= 165)");
    if (!A_dev || !r_dev || !dx_dev || !status_dev) return set_error(DDSG_ERR_ARG, "irbc_lu_solve: NULL argument");
    return lu_solve_masked(n, ns, A_dev, r_dev, nullptr, dx_dev, status_dev, 0x1p-46,
                           reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int irbc_newton(irbc_t *M, hdmr_t *policy, int64_t ns, const double *states_dev, double *sol_dev,
                           int max_it, double tol, int32_t *iters_dev, int32_t *status_dev,
                           double *resnorm_dev, int precision, int form, ddsg_stream_t stream) {
    if (!M || !policy || ns < 0 || max_it < 0 || !(tol > 0.0))
        return set_error(DDSG_ERR_ARG, "irbc_newton: bad argument");
    if (ns == 0) return DDSG_OK;
    if ((ns > 0) && (!states_dev || !sol_dev)) return set_error(DDSG_ERR_ARG, "irbc_newton: NULL states or solution");
    const int N = M->p.N, n = M->irreversible ? 2 * N + 1 : N + 1, d = 2 * N;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // Newton buffers (separate from the residual workspace): r, J, dz, zt, rt, norms,
    // steps, flags, and the compacted working set (two copies of its states and
    // solutions, spare r and dz, slot indices)
    double *r = nullptr, *J = nullptr, *dz = nullptr, *zt = nullptr, *rt = nullptr;
    double *n2 = nullptr, *ninf = nullptr, *n2t = nullptr, *ninft = nullptr, *step = nullptr;
    int32_t *active = nullptr, *stat = nullptr;
    auto bytes = [&](size_t k) { return sizeof(double) * k; };
    auto rnd = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // sub-buffer sizes, each rounded to 256 bytes; the block is exactly their sum
    const size_t szv = rnd(bytes((size_t)ns * n)), szJ = rnd(bytes((size_t)ns * n * n)),
                 szs = rnd(bytes((size_t)ns)), szi = rnd(sizeof(int32_t) * (size_t)ns),
                 szS = rnd(bytes((size_t)ns * d)), szl = rnd(sizeof(int64_t) * (size_t)ns);
    const size_t tot = 4 * szv + szJ + 5 * szs + 4 * szi + 2 * szS + 4 * szv + szl;
    if (tot > M->nws_bytes) {
        cudaFree(M->nws);
        M->nws = nullptr;
        M->nws_bytes = 0;
        if (dev_alloc(&M->nws, tot) != cudaSuccess) {
            cudaGetLastError();
            return set_error(DDSG_ERR_OOM, "irbc_newton: buffers unavailable");
        }
        M->nws_bytes = tot;
    }
    void *blk = M->nws;
    unsigned char *p = static_cast<unsigned char *>(blk);
    auto take = [&](size_t rounded) { unsigned char *q = p; p += rounded; return q; };
    r = (double *)take(szv);
    rt = (double *)take(szv);
    dz = (double *)take(szv);
    zt = (double *)take(szv);
    J = (double *)take(szJ);
    n2 = (double *)take(szs);
    ninf = (double *)take(szs);
    n2t = (double *)take(szs);
    ninft = (double *)take(szs);
    step = (double *)take(szs);
    active = (int32_t *)take(szi);
    stat = (int32_t *)take(szi);
    int32_t *accd = (int32_t *)take(szi);
    int32_t *kidx_d = (int32_t *)take(szi);
    double *Sw[2] = {(double *)take(szS), (double *)take(szS)};
    double *Zw[2] = {(double *)take(szv), (double *)take(szv)};
    double *r2 = (double *)take(szv), *dz2 = (double *)take(szv);
    int64_t *widx_d = (int64_t *)take(szl);
    if ((size_t)(p - static_cast<unsigned char *>(blk)) != tot)
        return set_error(DDSG_ERR_STATE, "irbc_newton: internal buffer layout mismatch");
    std::vector<double> h_n2(ns), h_ninf(ns), h_n2t(ns), h_step(ns), h_res(ns, 0.0);
    std::vector<int32_t> h_active(ns, 1), h_iters(ns, 0), h_stat(ns, 1);   // 1 = max-iter until converged
    int rc = DDSG_OK;
    auto fail_cuda = [&](cudaError_t e) { rc = set_error(DDSG_ERR_CUDA, cudaGetErrorString(e)); };
    // The working set: slot k holds state widx[k]. It starts as the caller's
    // arrays; once at most 3/4 of its slots are still iterating, the live ones
    // are gathered into contiguous slots (states, solution, residual, step), so
    // converged states cost nothing in later iterations. Per-state arithmetic
    // does not depend on the slot, so the results are those of the full batch.
    std::vector<int64_t> widx(ns);
    for (int64_t s = 0; s < ns; ++s) widx[s] = s;
    int64_t nw = ns;
    const double *S = states_dev;
    double *Z = sol_dev;
    int wb = 0;
    bool own = false;   // Z is a working copy (scattered back at the end)
    // The residual, its norms and the Jacobian at the accepted points come out
    // of the last line-search evaluation (it is evaluated with the Jacobian), so
    // an iteration after a step reuses them instead of evaluating again.
    bool have_next = false;
    for (int it = 0; it <= max_it && rc == DDSG_OK; ++it) {
        const unsigned nb = (unsigned)((nw + 255) / 256);
        if (have_next) {
            std::swap(r, rt);
            std::swap(n2, n2t);
            std::swap(ninf, ninft);
        } else {
            rc = euler_residual(M, policy, nw, S, Z, r, it < max_it ? J : nullptr, nullptr, precision, form, stream);
            if (rc) break;
            Tracer::Scope ts(&M->tr, 5, st);
            norms_kernel<<<nb, 256, 0, st>>>(n, nw, r, n2, ninf);
        }
        have_next = false;
        cudaError_t e = cudaMemcpyAsync(h_n2.data(), n2, bytes(nw), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_ninf.data(), ninf, bytes(nw), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { fail_cuda(e); break; }
        int64_t live = 0;
        std::vector<int32_t> act(nw);
        for (int64_t k = 0; k < nw; ++k) {
            const int64_t s = widx[k];
            h_res[s] = h_ninf[k];
            if (h_active[s] && h_ninf[k] <= tol) {
                h_active[s] = 0;
                h_stat[s] = 0;
            }
            act[k] = h_active[s];
            live += act[k];
        }
        if (live == 0 || it == max_it) break;
        // Newton step dz = -J^-1 r for the live slots
        e = cudaMemsetAsync(stat, 0, sizeof(int32_t) * nw, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(active, act.data(), sizeof(int32_t) * nw, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { fail_cuda(e); break; }
        {
            Tracer::Scope ts(&M->tr, 4, st);
            // F32C: the Jacobian's derivative sums are FP32, so the step is refined
            // to 2^-30 of its size; FP64: to FP64 accuracy
            rc = lu_solve_masked(n, nw, J, r, active, dz, stat, precision == DDSG_F32C ? 0x1p-30 : 0x1p-46, st);
        }
        if (rc) break;
        std::vector<int32_t> h_lu(nw);
        e = cudaMemcpyAsync(h_lu.data(), stat, sizeof(int32_t) * nw, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { fail_cuda(e); break; }
        for (int64_t k = 0; k < nw; ++k) {
            const int64_t s = widx[k];
            if (h_active[s] && h_lu[k] == 2) {
                h_active[s] = 0;
                h_stat[s] = 2;   // singular Jacobian
                --live;
            }
        }
        if (live > 0 && live * 4 <= nw * 3) {
            // compact: the live slots, in order, into the other working buffers
            std::vector<int32_t> kidx;
            std::vector<int64_t> nidx;
            std::vector<double> n2c;
            kidx.reserve(live);
            nidx.reserve(live);
            n2c.reserve(live);
            for (int64_t k = 0; k < nw; ++k)
                if (h_active[widx[k]]) {
                    kidx.push_back((int32_t)k);
                    nidx.push_back(widx[k]);
                    n2c.push_back(h_n2[k]);
                }
            Tracer::Scope ts(&M->tr, 5, st);
            if (own) {   // the leaving slots' solutions go back first
                e = cudaMemcpyAsync(widx_d, widx.data(), sizeof(int64_t) * nw, cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess) {
                    scatter_rows_kernel<<<(unsigned)((nw * n + 255) / 256), 256, 0, st>>>(nw, n, widx_d, Z, sol_dev);
                    e = cudaGetLastError();
                }
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(kidx_d, kidx.data(), sizeof(int32_t) * live, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) {
                const unsigned gs = (unsigned)((live * d + 255) / 256), gv = (unsigned)((live * n + 255) / 256);
                double *Sn = Sw[wb ^ 1], *Zn = Zw[wb ^ 1];
                gather_rows_kernel<<<gs, 256, 0, st>>>(live, d, kidx_d, S, Sn);
                gather_rows_kernel<<<gv, 256, 0, st>>>(live, n, kidx_d, Z, Zn);
                gather_rows_kernel<<<gv, 256, 0, st>>>(live, n, kidx_d, r, r2);
                gather_rows_kernel<<<gv, 256, 0, st>>>(live, n, kidx_d, dz, dz2);
                e = cudaGetLastError();
                S = Sn;
                Z = Zn;
                std::swap(r, r2);
                std::swap(dz, dz2);
                wb ^= 1;
                own = true;
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // kidx outlives its copy
            if (e != cudaSuccess) { fail_cuda(e); break; }
            widx.swap(nidx);
            nw = live;
            std::copy(n2c.begin(), n2c.end(), h_n2.begin());
        }
        for (int64_t k = 0; k < nw; ++k) h_step[k] = 1.0;
        // backtracking on ||r||_2: halve per state until the norm decreases
        std::vector<int32_t> pending(nw);
        for (int64_t k = 0; k < nw; ++k) pending[k] = h_active[widx[k]];
        const unsigned nbw = (unsigned)((nw + 255) / 256);
        for (int ls = 0; ls < 12; ++ls) {
            int64_t np = 0;
            for (int64_t k = 0; k < nw; ++k) np += pending[k];
            if (np == 0) break;
            e = cudaMemcpyAsync(active, pending.data(), sizeof(int32_t) * nw, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(step, h_step.data(), bytes(nw), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { fail_cuda(e); break; }
            {
                Tracer::Scope ts(&M->tr, 5, st);
                trial_kernel<<<(unsigned)((nw * n + 255) / 256), 256, 0, st>>>(n, nw, Z, dz, step, active, zt);
            }
            // with the Jacobian when the next iteration may take a step: after the
            // last round every slot's trial point is its accepted point
            rc = euler_residual(M, policy, nw, S, zt, rt, it + 1 < max_it ? J : nullptr, nullptr, precision, form,
                                stream);
            if (rc) break;
            have_next = true;
            {
                Tracer::Scope ts(&M->tr, 5, st);
                norms_kernel<<<nbw, 256, 0, st>>>(n, nw, rt, n2t, ninft);
            }
            e = cudaMemcpyAsync(h_n2t.data(), n2t, bytes(nw), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { fail_cuda(e); break; }
            std::vector<int32_t> acc(nw, 0);
            int64_t na = 0;
            for (int64_t k = 0; k < nw; ++k) {
                if (!pending[k]) continue;
                if (h_n2t[k] < h_n2[k] || ls == 11) {
                    acc[k] = 1;
                    pending[k] = 0;
                    ++na;
                } else {
                    h_step[k] *= 0.5;
                }
            }
            if (na) {
                // copy accepted trial points into the solution (acc is read before the
                // stream reaches the next host synchronization, so it must outlive the copy)
                e = cudaMemcpyAsync(accd, acc.data(), sizeof(int32_t) * nw, cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess) {
                    Tracer::Scope ts(&M->tr, 5, st);
                    accept_kernel<<<(unsigned)((nw * n + 255) / 256), 256, 0, st>>>(n, nw, accd, zt, Z);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) { fail_cuda(e); break; }
            }
        }
        for (int64_t s = 0; s < ns; ++s)
            if (h_active[s]) h_iters[s] = it + 1;
    }
    if (rc == DDSG_OK && own) {   // the working copies' solutions back to the caller's array
        cudaError_t e = cudaMemcpyAsync(widx_d, widx.data(), sizeof(int64_t) * nw, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            scatter_rows_kernel<<<(unsigned)((nw * n + 255) / 256), 256, 0, st>>>(nw, n, widx_d, Z, sol_dev);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) fail_cuda(e);
    }
    if (rc == DDSG_OK) {
        cudaError_t e = cudaSuccess;
        if (iters_dev) e = cudaMemcpyAsync(iters_dev, h_iters.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && status_dev)
            e = cudaMemcpyAsync(status_dev, h_stat.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && resnorm_dev)
            e = cudaMemcpyAsync(resnorm_dev, h_res.data(), bytes(ns), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) fail_cuda(e);
    }
    return rc;
}

extern "C" int irbc_profile(irbc_t *M, int enable) {
    if (!M) return set_error(DDSG_ERR_ARG, "irbc_profile: NULL model");
    M->tr.on = enable != 0;
    return DDSG_OK;
}

extern "C" int irbc_profile_read(irbc_t *M, double *ms, int64_t *launches, int reset) {
    if (!M) return set_error(DDSG_ERR_ARG, "irbc_profile_read: NULL model");
    M->tr.read(ms, launches, reset != 0);
    return DDSG_OK;
}

namespace ddsg {
// Check word of this module, read and cleared (all bits set if it cannot be read).
unsigned long long check_word_take_irbc() {
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
