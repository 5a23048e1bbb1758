// ddsg_mlp.cu -- warm-start network: a GELU MLP trained and evaluated with
// hand-written BF16 tensor-core GEMMs (mma.sync m16n8k16, FP32 accumulate).
//
// The network proposes Newton initial guesses for the IRBC step; the paper
// has no network -- the interpolant and the Newton solve stay the judges.
//
// Layout: every width is padded to a multiple of 64 with zeros (weights,
// biases, activations); batches are padded to a multiple of 64 rows whose
// inputs and loss gradients are zero. Master weights and Adam moments are
// FP32; GEMM operands are BF16 copies (W and its transpose).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ddsg_alloc.h"
#include "ddsg_internal.h"
#include "ddsg_io.h"

using namespace ddsg;

namespace {

constexpr int BM = 64, BN = 64, BK = 32, PADK = 8;
constexpr int GEMM_THREADS = 128;

enum { EPI_STORE = 0, EPI_HIDDEN = 1, EPI_LAST = 2, EPI_GELU_BWD = 3 };

struct Epi {
    float *f;            // FP32 output (STORE, LAST: result; GELU_BWD: dZ)
    int ldf;
    float *z;            // HIDDEN: pre-activation (nullable)
    int ldz;
    __nv_bfloat16 *h;    // HIDDEN: GELU(z) as BF16; GELU_BWD: dZ as BF16
    int ldh;
    const float *bias;   // HIDDEN, LAST
    const float *zp;     // GELU_BWD: pre-activation of the layer below
    int ldzp;
    int64_t zstride;     // STORE with split K: split z writes f + z * zstride
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[M x N] = op(A)[M x K] * op(B)[N x K]^T. TA: A is stored K x M (element
// (m, k) at A[k*lda + m]); otherwise M x K. TB likewise for B (N x K or K x N).
// M, N multiples of 64 and K a multiple of 32 (the callers pad). Split K: block
// z of the grid's third dimension covers k in [z*kchunk, min(K, (z+1)*kchunk))
// and (STORE only) writes its partial product at f + z * zstride.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16 *__restrict__ A,
                                                                 int lda, const __nv_bfloat16 *__restrict__ B, int ldb,
                                                                 Epi e, int kchunk) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PADK];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PADK];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int wm = warp >> 1, wn = warp & 1;  // 2 x 2 warps, 32 x 32 each
    const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        for (int idx = tid; idx < BM * BK; idx += GEMM_THREADS) {
            int r, c;
            if (TA) { r = idx % BM; c = idx / BM; } else { r = idx / BK; c = idx % BK; }
            const int m = bm + r, k = k0 + c;
            __nv_bfloat16 v = __float2bfloat16(0.f);
            if (m < M && k < ke) v = TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
            As[r][c] = v;
        }
        for (int idx = tid; idx < BN * BK; idx += GEMM_THREADS) {
            int r, c;
            if (TB) { r = idx % BN; c = idx / BN; } else { r = idx / BK; c = idx % BK; }
            const int n = bn + r, k = k0 + c;
            __nv_bfloat16 v = __float2bfloat16(0.f);
            if (n < N && k < ke) v = TB ? B[(int64_t)k * ldb + n] : B[(int64_t)n * ldb + k];
            Bs[r][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r0 = wm * 32 + i * 16 + g;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r0][kk + 2 * t]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r0 + 8][kk + 2 * t]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r0][kk + 8 + 2 * t]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r0 + 8][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n0 = wn * 32 + j * 8 + g;
                bf[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[n0][kk + 2 * t]);
                bf[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[n0][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(acc[i][j], af[i][0], af[i][1], af[i][2], af[i][3], bf[j][0], bf[j][1]);
        }
        __syncthreads();
    }
    // epilogue: acc[i][j][r] -> (row, col)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = bm + wm * 32 + i * 16 + g + (r >= 2 ? 8 : 0);
                const int col = bn + wn * 32 + j * 8 + 2 * t + (r & 1);
                if (row >= M || col >= N) continue;
                const float v = acc[i][j][r];
                if (EPI == EPI_STORE) {
                    e.f[(int64_t)blockIdx.z * e.zstride + (int64_t)row * e.ldf + col] = v;
                } else if (EPI == EPI_HIDDEN) {
                    const float z = v + e.bias[col];
                    if (e.z) e.z[(int64_t)row * e.ldz + col] = z;
                    e.h[(int64_t)row * e.ldh + col] = __float2bfloat16(gelu_f(z));
                } else if (EPI == EPI_LAST) {
                    e.f[(int64_t)row * e.ldf + col] = v + e.bias[col];
                } else {
                    const float dz = v * gelu_grad_f(e.zp[(int64_t)row * e.ldzp + col]);
                    e.f[(int64_t)row * e.ldf + col] = dz;
                    e.h[(int64_t)row * e.ldh + col] = __float2bfloat16(dz);
                }
            }
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                 const Epi &e, cudaStream_t st, int splits = 1, int kchunk = 0) {
    dim3 grid((unsigned)(N / BN), (unsigned)(M / BM), (unsigned)splits);
    gemm_bf16_kernel<TA, TB, EPI><<<grid, GEMM_THREADS, 0, st>>>(M, N, K, A, lda, B, ldb, e, splits > 1 ? kchunk : K);
    return cudaGetLastError();
}

// Split of the batch dimension (K of the weight-gradient GEMM) so that the
// (Po/64) x (Pi/64) output tiles times the splits fill the SMs about twice;
// chunks are multiples of BK.
void grad_split(int64_t Bp, int Po, int Pi, int &splits, int &kchunk) {
    const int tiles = (Po / BM) * (Pi / BN);
    const int want = std::max(1, (2 * 152 + tiles - 1) / tiles);
    const int64_t kmax = std::max<int64_t>(1, Bp / BK);
    const int s = (int)std::min<int64_t>(want, kmax);
    kchunk = (int)(((Bp + s - 1) / s + BK - 1) / BK * BK);
    splits = (int)((Bp + kchunk - 1) / kchunk);
}

// x (B x n0, FP64 physical) -> (x - shift) * scale as BF16 in B_pad x P0 (zero padding)
__global__ void mlp_input_kernel(int64_t B, int64_t Bp, int n0, int P0, const double *__restrict__ x,
                                 const double *__restrict__ shift, const double *__restrict__ scale,
                                 __nv_bfloat16 *__restrict__ X) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Bp * P0) return;
    const int64_t b = e / P0;
    const int c = (int)(e - b * P0);
    float v = 0.f;
    if (b < B && c < n0) v = (float)((x[b * n0 + c] - shift[c]) * scale[c]);
    X[e] = __float2bfloat16(v);
}

// dY = 2 (Y - T) / (B m) on the normalized targets; loss += sum (Y - T)^2 / (B m)
__global__ void mlp_loss_kernel(int64_t B, int64_t Bp, int m, int PL, const float *__restrict__ Y,
                                const double *__restrict__ y, const double *__restrict__ shift,
                                const double *__restrict__ scale, float *__restrict__ dY,
                                __nv_bfloat16 *__restrict__ dYb, double *__restrict__ loss) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (e < Bp * PL) {
        const int64_t b = e / PL;
        const int c = (int)(e - b * PL);
        float g = 0.f;
        if (b < B && c < m) {
            const double tgt = (y[b * m + c] - shift[c]) * scale[c];
            const double diff = (double)Y[e] - tgt;
            l = diff * diff / ((double)B * m);
            g = (float)(2.0 * diff / ((double)B * m));
        }
        dY[e] = g;
        dYb[e] = __float2bfloat16(g);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// column sums of dZ (Bp x P): one thread per column, rows in order
// Partial column sums of dZ (Bp x P) over the rows [z*kchunk, min(Bp, (z+1)*kchunk))
// of block z: 32 columns x 8 row lanes per block, part[z*P + c].
__global__ void colsum_part_kernel(int64_t Bp, int P, int kchunk, const float *__restrict__ dZ,
                                   float *__restrict__ part) {
    __shared__ float s[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    const int64_t b0 = (int64_t)blockIdx.y * kchunk, b1 = min(Bp, b0 + kchunk);
    float acc = 0.f;
    if (c < P)
        for (int64_t b = b0 + ty; b < b1; b += 8) acc += dZ[b * P + c];
    s[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && c < P) {
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) t += s[i][tx];
        part[(int64_t)blockIdx.y * P + c] = t;
    }
}

// out[i] = sum over z of part[z*n + i], in z order (deterministic)
__global__ void splitk_reduce_kernel(int splits, int64_t n, const float *__restrict__ part, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * n + i];
    out[i] = s;
}

// Adam on one parameter tensor (FP32 master), refreshing its BF16 copy and,
// for weights, the transposed BF16 copy (rows x cols -> cols x rows).
__global__ void adam_kernel(int64_t n, int rows, int cols, float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ mo, float *__restrict__ ve, float lr, float b1, float b2, float eps,
                            float c1, float c2, __nv_bfloat16 *__restrict__ pb, __nv_bfloat16 *__restrict__ pbt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gr = g[e];
    const float m1 = b1 * mo[e] + (1.f - b1) * gr;
    const float v1 = b2 * ve[e] + (1.f - b2) * gr * gr;
    mo[e] = m1;
    ve[e] = v1;
    const float np = p[e] - lr * (m1 / c1) / (sqrtf(v1 / c2) + eps);
    p[e] = np;
    if (pb) pb[e] = __float2bfloat16(np);
    if (pbt) {
        const int r = (int)(e / cols), c = (int)(e - (int64_t)r * cols);
        pbt[(int64_t)c * rows + r] = __float2bfloat16(np);
    }
}

__global__ void to_bf16_kernel(int64_t n, int rows, int cols, const float *__restrict__ p,
                               __nv_bfloat16 *__restrict__ pb, __nv_bfloat16 *__restrict__ pbt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const __nv_bfloat16 v = __float2bfloat16(p[e]);
    if (pb) pb[e] = v;
    if (pbt) {
        const int r = (int)(e / cols), c = (int)(e - (int64_t)r * cols);
        pbt[(int64_t)c * rows + r] = v;
    }
}

// y (B x m, FP64) = Y_normalized / scale + shift
__global__ void mlp_output_kernel(int64_t B, int m, int PL, const float *__restrict__ Y,
                                  const double *__restrict__ shift, const double *__restrict__ scale,
                                  double *__restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * m) return;
    const int64_t b = e / m;
    const int c = (int)(e - b * m);
    y[e] = (double)Y[b * PL + c] / scale[c] + shift[c];
}

inline int pad64(int n) { return (n + 63) & ~63; }
inline int64_t pad64l(int64_t n) { return (n + 63) & ~63ll; }
inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

struct mlp {
    int L = 0;
    std::vector<int> n, P;        // logical / padded widths, L+1 each
    int device = -1;
    // per layer device tensors
    std::vector<float *> W, b, gW, gb, mW, vW, mb, vb;
    std::vector<__nv_bfloat16 *> Wb, WbT;
    double *in_shift = nullptr, *in_scale = nullptr, *out_shift = nullptr, *out_scale = nullptr;
    std::vector<float> init;      // packed FP32 parameters before upload
    std::vector<float> init_m, init_v;   // packed Adam moments before upload (empty: zero)
    std::vector<double> norm;     // in_shift, in_scale, out_shift, out_scale
    int64_t step = 0;
    // batch workspace
    int64_t cap = 0;
    void *ws = nullptr;
    double *loss = nullptr;
    Tracer tr;                    // kinds: 0 gemm forward, 1 gemm backward, 2 loss/aux, 3 adam
};

namespace {

// Device parameter buffers (not the batch workspace) back to nothing held.
void release_params(mlp *M) {
    for (int l = 0; l < (int)M->W.size(); ++l) {
        cudaFree(M->W[l]); cudaFree(M->b[l]); cudaFree(M->gW[l]); cudaFree(M->gb[l]);
        cudaFree(M->mW[l]); cudaFree(M->vW[l]); cudaFree(M->mb[l]); cudaFree(M->vb[l]);
        cudaFree(M->Wb[l]); cudaFree(M->WbT[l]);
    }
    M->W.clear(); M->b.clear(); M->gW.clear(); M->gb.clear(); M->mW.clear();
    M->vW.clear(); M->mb.clear(); M->vb.clear(); M->Wb.clear(); M->WbT.clear();
    cudaFree(M->in_shift); cudaFree(M->in_scale); cudaFree(M->out_shift); cudaFree(M->out_scale);
    cudaFree(M->loss);
    M->in_shift = M->in_scale = M->out_shift = M->out_scale = nullptr;
    M->loss = nullptr;
}

int mlp_bind(mlp *M) {
    if (M->device >= 0) return DDSG_OK;
    release_params(M);   // what an earlier failed bind left behind
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(DDSG_ERR_CUDA, "mlp: no CUDA device");
    auto alloc = [](void **p, size_t b) { return dev_alloc(p, b) == cudaSuccess && cudaMemset(*p, 0, b) == cudaSuccess; };
    const int L = M->L;
    M->W.assign(L, nullptr); M->b.assign(L, nullptr); M->gW.assign(L, nullptr); M->gb.assign(L, nullptr);
    M->mW.assign(L, nullptr); M->vW.assign(L, nullptr); M->mb.assign(L, nullptr); M->vb.assign(L, nullptr);
    M->Wb.assign(L, nullptr); M->WbT.assign(L, nullptr);
    size_t off = 0;
    for (int l = 0; l < L; ++l) {
        const int Pi = M->P[l], Po = M->P[l + 1];
        const size_t nw = (size_t)Pi * Po;
        bool ok = alloc((void **)&M->W[l], nw * 4) && alloc((void **)&M->gW[l], nw * 4) &&
                  alloc((void **)&M->mW[l], nw * 4) && alloc((void **)&M->vW[l], nw * 4) &&
                  alloc((void **)&M->b[l], Po * 4) && alloc((void **)&M->gb[l], Po * 4) &&
                  alloc((void **)&M->mb[l], Po * 4) && alloc((void **)&M->vb[l], Po * 4) &&
                  alloc((void **)&M->Wb[l], nw * 2) && alloc((void **)&M->WbT[l], nw * 2);
        if (!ok) return set_error(DDSG_ERR_OOM, "mlp: parameter allocation failed");
        // scatter the packed logical parameters (and saved Adam moments) into the padded layout
        const int ni = M->n[l], no = M->n[l + 1];
        auto upload = [&](const std::vector<float> &src, float *dW, float *db) {
            std::vector<float> w(nw, 0.f), bb(Po, 0.f);
            for (int r = 0; r < no; ++r)
                for (int c = 0; c < ni; ++c) w[(size_t)r * Pi + c] = src[off + (size_t)r * ni + c];
            for (int r = 0; r < no; ++r) bb[r] = src[off + (size_t)no * ni + r];
            return cudaMemcpy(dW, w.data(), nw * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
                   cudaMemcpy(db, bb.data(), Po * 4, cudaMemcpyHostToDevice) == cudaSuccess;
        };
        bool up = upload(M->init, M->W[l], M->b[l]);
        if (up && !M->init_m.empty()) up = upload(M->init_m, M->mW[l], M->mb[l]) && upload(M->init_v, M->vW[l], M->vb[l]);
        off += (size_t)no * ni + no;
        if (!up) return set_error(DDSG_ERR_CUDA, "mlp: parameter upload failed");
        to_bf16_kernel<<<nblk(nw), 256>>>((int64_t)nw, Po, Pi, M->W[l], M->Wb[l], M->WbT[l]);
        if (cudaGetLastError() != cudaSuccess) return set_error(DDSG_ERR_CUDA, "mlp: conversion failed");
    }
    const int n0 = M->n[0], nL = M->n[L];
    if (!alloc((void **)&M->in_shift, n0 * 8) || !alloc((void **)&M->in_scale, n0 * 8) ||
        !alloc((void **)&M->out_shift, nL * 8) || !alloc((void **)&M->out_scale, nL * 8) ||
        !alloc((void **)&M->loss, 8))
        return set_error(DDSG_ERR_OOM, "mlp: allocation failed");
    const double *nrm = M->norm.data();
    if (cudaMemcpy(M->in_shift, nrm, n0 * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(M->in_scale, nrm + n0, n0 * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(M->out_shift, nrm + 2 * n0, nL * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(M->out_scale, nrm + 2 * n0 + nL, nL * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return set_error(DDSG_ERR_CUDA, "mlp: normalization upload failed");
    if (cudaDeviceSynchronize() != cudaSuccess) return set_error(DDSG_ERR_CUDA, "mlp: setup failed");
    M->device = dev;
    return DDSG_OK;
}

// Batch workspace for Bp rows: X_0..X_{L-1} (BF16), Z_0..Z_{L-2} (FP32),
// Y (FP32), dZ ping-pong (FP32 + BF16).
struct WsView {
    std::vector<__nv_bfloat16 *> X;
    std::vector<float *> Z;
    float *Y;
    float *dZ[2];
    __nv_bfloat16 *dZb[2];
    float *split;   // split-K partials of one layer's weight and bias gradients
};

int mlp_ws(mlp *M, int64_t Bp, WsView &v) {
    const int L = M->L;
    int Pmax = 0;
    for (int p : M->P) Pmax = std::max(Pmax, p);
    auto rnd = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t need = 0;
    for (int l = 0; l < L; ++l) need += rnd((size_t)Bp * M->P[l] * 2);
    for (int l = 0; l + 1 < L; ++l) need += rnd((size_t)Bp * M->P[l + 1] * 4);
    need += rnd((size_t)Bp * M->P[L] * 4);
    need += 2 * rnd((size_t)Bp * Pmax * 4) + 2 * rnd((size_t)Bp * Pmax * 2);
    size_t split_floats = 0;
    for (int l = 0; l < L; ++l) {
        int s = 1, kc = 0;
        grad_split(Bp, M->P[l + 1], M->P[l], s, kc);
        split_floats = std::max(split_floats, (size_t)s * ((size_t)M->P[l + 1] * M->P[l] + M->P[l + 1]));
    }
    need += rnd(split_floats * 4);
    if (Bp > M->cap) {
        cudaFree(M->ws);
        M->ws = nullptr;
        M->cap = 0;
        if (dev_alloc(&M->ws, need) != cudaSuccess) {
            cudaGetLastError();
            return set_error(DDSG_ERR_OOM, "mlp: batch workspace unavailable");
        }
        M->cap = Bp;
    }
    unsigned char *p = static_cast<unsigned char *>(M->ws);
    auto take = [&](size_t b) { unsigned char *q = p; p += rnd(b); return q; };
    v.X.resize(L);
    v.Z.resize(L);
    for (int l = 0; l < L; ++l) v.X[l] = (__nv_bfloat16 *)take((size_t)Bp * M->P[l] * 2);
    for (int l = 0; l + 1 < L; ++l) v.Z[l] = (float *)take((size_t)Bp * M->P[l + 1] * 4);
    v.Y = (float *)take((size_t)Bp * M->P[L] * 4);
    for (int i = 0; i < 2; ++i) v.dZ[i] = (float *)take((size_t)Bp * Pmax * 4);
    for (int i = 0; i < 2; ++i) v.dZb[i] = (__nv_bfloat16 *)take((size_t)Bp * Pmax * 2);
    v.split = (float *)take(split_floats * 4);
    return DDSG_OK;
}

// forward pass through all layers; keepZ stores pre-activations for training
cudaError_t mlp_forward(mlp *M, int64_t B, int64_t Bp, const double *x, WsView &v, bool keepZ, cudaStream_t st) {
    const int L = M->L;
    {
        Tracer::Scope ts(&M->tr, 2, st);
        mlp_input_kernel<<<nblk(Bp * M->P[0]), 256, 0, st>>>(B, Bp, M->n[0], M->P[0], x, M->in_shift, M->in_scale,
                                                             v.X[0]);
    }
    cudaError_t e = cudaGetLastError();
    Tracer::Scope ts(&M->tr, 0, st);
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        Epi ep = {};
        ep.bias = M->b[l];
        if (l + 1 < L) {
            ep.z = keepZ ? v.Z[l] : nullptr;
            ep.ldz = M->P[l + 1];
            ep.h = v.X[l + 1];
            ep.ldh = M->P[l + 1];
            e = gemm<false, false, EPI_HIDDEN>((int)Bp, M->P[l + 1], M->P[l], v.X[l], M->P[l], M->Wb[l], M->P[l], ep, st);
        } else {
            ep.f = v.Y;
            ep.ldf = M->P[L];
            e = gemm<false, false, EPI_LAST>((int)Bp, M->P[L], M->P[l], v.X[l], M->P[l], M->Wb[l], M->P[l], ep, st);
        }
    }
    return e;
}

}  // namespace

extern "C" int mlp_create(int nlayers, const int32_t *sizes, const float *params_host, uint64_t seed,
                          mlp_t **out) {
    if (!sizes || !out || nlayers < 1 || nlayers > 16) return set_error(DDSG_ERR_ARG, "mlp_create: bad argument");
    mlp *M = new (std::nothrow) mlp();
    if (!M) return set_error(DDSG_ERR_OOM, "mlp_create: host allocation failed");
    M->L = nlayers;
    size_t np = 0;
    for (int l = 0; l <= nlayers; ++l) {
        if (sizes[l] < 1 || sizes[l] > 8192) { delete M; return set_error(DDSG_ERR_ARG, "mlp_create: layer width out of range"); }
        M->n.push_back(sizes[l]);
        M->P.push_back(pad64(sizes[l]));
    }
    for (int l = 0; l < nlayers; ++l) np += (size_t)sizes[l] * sizes[l + 1] + sizes[l + 1];
    M->init.resize(np);
    if (params_host) {
        std::copy(params_host, params_host + np, M->init.begin());
    } else {
        // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from SplitMix64 (seed, counter); zero biases
        uint64_t ctr = 0;
        size_t off = 0;
        for (int l = 0; l < nlayers; ++l) {
            const double bound = 1.0 / sqrt((double)sizes[l]);
            for (size_t e = 0; e < (size_t)sizes[l] * sizes[l + 1]; ++e) {
                const uint64_t z = mix64(seed + (++ctr) * 0x9E3779B97F4A7C15ull);
                const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
                M->init[off++] = (float)((2.0 * u - 1.0) * bound);
            }
            for (int e = 0; e < sizes[l + 1]; ++e) M->init[off++] = 0.f;
        }
    }
    M->norm.assign(2 * sizes[0] + 2 * sizes[nlayers], 0.0);
    for (int c = 0; c < sizes[0]; ++c) M->norm[sizes[0] + c] = 1.0;
    for (int c = 0; c < sizes[nlayers]; ++c) M->norm[2 * sizes[0] + sizes[nlayers] + c] = 1.0;
    *out = M;
    return DDSG_OK;
}

extern "C" int mlp_destroy(mlp_t *M) {
    if (!M) return DDSG_OK;
    release_params(M);
    cudaFree(M->ws);
    delete M;
    return DDSG_OK;
}

extern "C" int mlp_set_normalization(mlp_t *M, const double *in_shift, const double *in_scale,
                                     const double *out_shift, const double *out_scale) {
    if (!M || !in_shift || !in_scale || !out_shift || !out_scale) return set_error(DDSG_ERR_ARG, "mlp_set_normalization: NULL argument");
    if (M->device >= 0) return set_error(DDSG_ERR_STATE, "mlp_set_normalization: set it before the first GPU call");
    const int n0 = M->n[0], nL = M->n[M->L];
    std::copy(in_shift, in_shift + n0, M->norm.begin());
    std::copy(in_scale, in_scale + n0, M->norm.begin() + n0);
    std::copy(out_shift, out_shift + nL, M->norm.begin() + 2 * n0);
    std::copy(out_scale, out_scale + nL, M->norm.begin() + 2 * n0 + nL);
    return DDSG_OK;
}

extern "C" int mlp_infer(mlp_t *M, int64_t B, const double *x_dev, double *y_dev, ddsg_stream_t stream) {
    if (!M || B < 0 || (B > 0 && (!x_dev || !y_dev))) return set_error(DDSG_ERR_ARG, "mlp_infer: bad argument");
    if (B == 0) return DDSG_OK;
    int rc = mlp_bind(M);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t chunk = 65536;
    {
        WsView v0;   // size the workspace once for the largest chunk (no reallocation between chunks)
        if ((rc = mlp_ws(M, pad64l(std::min(chunk, B)), v0))) return rc;
    }
    for (int64_t b0 = 0; b0 < B; b0 += chunk) {
        const int64_t nb = std::min(chunk, B - b0);
        const int64_t Bp = pad64l(nb);
        WsView v;
        if ((rc = mlp_ws(M, Bp, v))) return rc;
        cudaError_t e = mlp_forward(M, nb, Bp, x_dev + b0 * M->n[0], v, false, st);
        if (e == cudaSuccess) {
            Tracer::Scope ts(&M->tr, 2, st);
            mlp_output_kernel<<<nblk(nb * M->n[M->L]), 256, 0, st>>>(nb, M->n[M->L], M->P[M->L], v.Y, M->out_shift,
                                                                     M->out_scale, y_dev + b0 * M->n[M->L]);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return set_error(DDSG_ERR_CUDA, cudaGetErrorString(e));
    }
    return DDSG_OK;
}

// One Adam step on a batch (B rows). loss_dev (nullable) receives the batch
// loss (FP64, device); the gradients of the step stay readable (mlp_get_grads).
extern "C" int mlp_train_step(mlp_t *M, int64_t B, const double *x_dev, const double *y_dev, float lr,
                              double *loss_dev, ddsg_stream_t stream) {
    if (!M || B <= 0 || !x_dev || !y_dev || !(lr >= 0.f)) return set_error(DDSG_ERR_ARG, "mlp_train_step: bad argument");
    if (B > (int64_t)1 << 24) return set_error(DDSG_ERR_ARG, "mlp_train_step: batch too large");
    int rc = mlp_bind(M);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t Bp = pad64l(B);
    WsView v;
    if ((rc = mlp_ws(M, Bp, v))) return rc;
    const int L = M->L;
    cudaError_t e = mlp_forward(M, B, Bp, x_dev, v, true, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->loss, 0, 8, st);
    if (e == cudaSuccess) {
        Tracer::Scope ts(&M->tr, 2, st);
        mlp_loss_kernel<<<nblk(Bp * M->P[L]), 256, 0, st>>>(B, Bp, M->n[L], M->P[L], v.Y, y_dev, M->out_shift,
                                                            M->out_scale, v.dZ[0], v.dZb[0], M->loss);
        e = cudaGetLastError();
    }
    // backward: layer l has input width P[l], output width P[l+1]; dZ[cur] holds dL/dZ_l
    int cur = 0;
    for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
        Tracer::Scope ts(&M->tr, 1, st);
        const int Pi = M->P[l], Po = M->P[l + 1];
        // gW = dZ^T (Po x Bp) * X_l (Bp x Pi): both operands stored transposed; the
        // batch (K) is split over blocks, partials summed in split order
        int splits = 1, kchunk = 0;
        grad_split(Bp, Po, Pi, splits, kchunk);
        const int64_t nw = (int64_t)Po * Pi;
        float *pw = v.split, *pb = v.split + (int64_t)splits * nw;
        Epi g = {};
        g.f = pw;
        g.ldf = Pi;
        g.zstride = nw;
        e = gemm<true, true, EPI_STORE>(Po, Pi, (int)Bp, v.dZb[cur], Po, v.X[l], Pi, g, st, splits, kchunk);
        if (e == cudaSuccess) {
            colsum_part_kernel<<<dim3((unsigned)((Po + 31) / 32), (unsigned)splits), 256, 0, st>>>(Bp, Po, kchunk,
                                                                                                v.dZ[cur], pb);
            splitk_reduce_kernel<<<nblk(nw), 256, 0, st>>>(splits, nw, pw, M->gW[l]);
            splitk_reduce_kernel<<<nblk(Po), 256, 0, st>>>(splits, Po, pb, M->gb[l]);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && l > 0) {
            Epi d = {};
            d.f = v.dZ[cur ^ 1];
            d.ldf = Pi;
            d.h = v.dZb[cur ^ 1];
            d.ldh = Pi;
            d.zp = v.Z[l - 1];
            d.ldzp = Pi;
            // dA = dZ (Bp x Po) * W (Po x Pi) = dZ * (W^T)^T with W^T stored Pi x Po
            e = gemm<false, false, EPI_GELU_BWD>((int)Bp, Pi, Po, v.dZb[cur], Po, M->WbT[l], Po, d, st);
            cur ^= 1;
        }
    }
    // Adam (bias corrections of step t)
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 - pow(0.9, (double)M->step)), c2 = (float)(1.0 - pow(0.999, (double)M->step));
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        Tracer::Scope ts(&M->tr, 3, st);
        const int Pi = M->P[l], Po = M->P[l + 1];
        const int64_t nw = (int64_t)Pi * Po;
        adam_kernel<<<nblk(nw), 256, 0, st>>>(nw, Po, Pi, M->W[l], M->gW[l], M->mW[l], M->vW[l], lr, b1, b2, eps, c1, c2,
                                             M->Wb[l], M->WbT[l]);
        adam_kernel<<<nblk(Po), 256, 0, st>>>(Po, 1, Po, M->b[l], M->gb[l], M->mb[l], M->vb[l], lr, b1, b2, eps, c1, c2,
                                             nullptr, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && loss_dev) e = cudaMemcpyAsync(loss_dev, M->loss, 8, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return set_error(DDSG_ERR_CUDA, cudaGetErrorString(e));
    return DDSG_OK;
}

// Packed logical parameters (per layer W row-major out x in, then b) or the
// gradients of the last train step, FP32, to the host. Synchronous.
// which: 0 parameters, 1 gradients of the last step, 2 / 3 Adam first / second moments;
// packed logical layout (per layer W row-major n_out x n_in, then b)
static int mlp_copy_out(mlp_t *M, int which, float *host) {
    if (!M || !host) return set_error(DDSG_ERR_ARG, "mlp: NULL argument");
    if (M->device < 0) {
        if (which == 1) return set_error(DDSG_ERR_STATE, "mlp_get_grads: no train step yet");
        const std::vector<float> &src = which == 0 ? M->init : (which == 2 ? M->init_m : M->init_v);
        if (src.empty()) std::fill(host, host + M->init.size(), 0.f);
        else std::copy(src.begin(), src.end(), host);
        return DDSG_OK;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return set_error(DDSG_ERR_CUDA, "mlp: synchronize failed");
    size_t off = 0;
    for (int l = 0; l < M->L; ++l) {
        const int Pi = M->P[l], Po = M->P[l + 1], ni = M->n[l], no = M->n[l + 1];
        std::vector<float> w((size_t)Pi * Po), bb(Po);
        const float *sW = which == 0 ? M->W[l] : which == 1 ? M->gW[l] : which == 2 ? M->mW[l] : M->vW[l];
        const float *sb = which == 0 ? M->b[l] : which == 1 ? M->gb[l] : which == 2 ? M->mb[l] : M->vb[l];
        if (cudaMemcpy(w.data(), sW, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(bb.data(), sb, bb.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return set_error(DDSG_ERR_CUDA, "mlp: copy failed");
        for (int r = 0; r < no; ++r)
            for (int c = 0; c < ni; ++c) host[off + (size_t)r * ni + c] = w[(size_t)r * Pi + c];
        off += (size_t)no * ni;
        for (int r = 0; r < no; ++r) host[off + r] = bb[r];
        off += no;
    }
    return DDSG_OK;
}

extern "C" int mlp_get_params(mlp_t *M, float *host) { return mlp_copy_out(M, 0, host); }
extern "C" int mlp_get_grads(mlp_t *M, float *host) { return mlp_copy_out(M, 1, host); }

// ---------------------------------------------------------------------------
// checkpoint / resume: one file per network (layout in ddsg_io.h):
//   i32 L, i32 sizes[L+1], i64 Adam step, f64 normalization[2 n_0 + 2 n_L],
//   f32 parameters[np], f32 Adam m[np], f32 Adam v[np] (packed logical layout)
// ---------------------------------------------------------------------------

constexpr char kMlpMagic[8] = {'D', 'D', 'S', 'G', 'M', 'L', 'P', 'N'};
constexpr uint32_t kMlpVersion = 1;

extern "C" int mlp_save(mlp_t *M, const char *path) {
    if (!M || !path) return set_error(DDSG_ERR_ARG, "mlp_save: NULL argument");
    const size_t np = M->init.size();
    std::vector<float> prm(np), mm(np), vv(np);
    int rc = mlp_copy_out(M, 0, prm.data());
    if (!rc) rc = mlp_copy_out(M, 2, mm.data());
    if (!rc) rc = mlp_copy_out(M, 3, vv.data());
    if (rc) return rc;
    std::vector<double> nrm = M->norm;
    if (M->device >= 0) {
        // the normalization lives on the device once bound (it cannot change then)
        const int n0 = M->n[0], nL = M->n[M->L];
        if (cudaMemcpy(nrm.data(), M->in_shift, n0 * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(nrm.data() + n0, M->in_scale, n0 * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(nrm.data() + 2 * n0, M->out_shift, nL * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(nrm.data() + 2 * n0 + nL, M->out_scale, nL * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return set_error(DDSG_ERR_CUDA, "mlp_save: copy failed");
    }
    io::Writer w;
    w.header(kMlpMagic, kMlpVersion);
    w.put1<int32_t>(M->L);
    for (int l = 0; l <= M->L; ++l) w.put1<int32_t>(M->n[l]);
    w.put1<int64_t>(M->step);
    w.put(nrm.data(), nrm.size());
    w.put(prm.data(), np);
    w.put(mm.data(), np);
    w.put(vv.data(), np);
    w.seal();
    if (!io::write_file(path, w.buf)) return set_error(DDSG_ERR_ARG, "mlp_save: write failed");
    return DDSG_OK;
}

extern "C" int mlp_load(const char *path, mlp_t **out) {
    if (!path || !out) return set_error(DDSG_ERR_ARG, "mlp_load: NULL argument");
    *out = nullptr;
    std::vector<unsigned char> buf;
    if (!io::read_file(path, buf)) return set_error(DDSG_ERR_ARG, "mlp_load: cannot open the file");
    io::Reader r{nullptr, nullptr};
    switch (io::open_body(buf, kMlpMagic, kMlpVersion, r)) {
        case 1: return set_error(DDSG_ERR_ARG, "mlp_load: not a network file");
        case 2: return set_error(DDSG_ERR_ARG, "mlp_load: unsupported file version");
        case 3: return set_error(DDSG_ERR_ARG, "mlp_load: checksum mismatch (truncated or corrupt file)");
        default: break;
    }
    int32_t L = 0;
    if (!r.get(&L, 1) || L < 1 || L > 16) return set_error(DDSG_ERR_ARG, "mlp_load: bad layer count");
    std::vector<int32_t> sizes(L + 1);
    int64_t step = 0;
    if (!r.get(sizes.data(), sizes.size()) || !r.get(&step, 1) || step < 0)
        return set_error(DDSG_ERR_ARG, "mlp_load: truncated header");
    size_t np = 0;
    for (int l = 0; l <= L; ++l)
        if (sizes[l] < 1 || sizes[l] > 8192) return set_error(DDSG_ERR_ARG, "mlp_load: layer width out of range");
    for (int l = 0; l < L; ++l) np += (size_t)sizes[l] * sizes[l + 1] + sizes[l + 1];
    std::vector<double> nrm(2 * (size_t)sizes[0] + 2 * (size_t)sizes[L]);
    std::vector<float> prm(np), mm(np), vv(np);
    if (!r.get(nrm.data(), nrm.size()) || !r.get(prm.data(), np) || !r.get(mm.data(), np) || !r.get(vv.data(), np) ||
        r.p != r.end)
        return set_error(DDSG_ERR_ARG, "mlp_load: file size does not match its header");
    mlp_t *M = nullptr;
    int rc = mlp_create(L, sizes.data(), prm.data(), 0, &M);
    if (rc) return rc;
    M->norm = nrm;
    M->step = step;
    M->init_m = std::move(mm);
    M->init_v = std::move(vv);
    *out = M;
    return DDSG_OK;
}

extern "C" int mlp_shape(const mlp_t *M, int32_t *nlayers, int32_t *sizes_host) {
    if (!M) return set_error(DDSG_ERR_ARG, "mlp_shape: NULL network");
    if (nlayers) *nlayers = M->L;
    if (sizes_host)
        for (int l = 0; l <= M->L; ++l) sizes_host[l] = M->n[l];
    return DDSG_OK;
}

extern "C" int64_t mlp_num_params(const mlp_t *M) {
    if (!M) return 0;
    int64_t np = 0;
    for (int l = 0; l < M->L; ++l) np += (int64_t)M->n[l] * M->n[l + 1] + M->n[l + 1];
    return np;
}

extern "C" int mlp_profile(mlp_t *M, int enable) {
    if (!M) return set_error(DDSG_ERR_ARG, "mlp_profile: NULL network");
    M->tr.on = enable != 0;
    return DDSG_OK;
}

extern "C" int mlp_profile_read(mlp_t *M, double *ms, int64_t *launches, int reset) {
    if (!M) return set_error(DDSG_ERR_ARG, "mlp_profile_read: NULL network");
    M->tr.read(ms, launches, reset != 0);
    return DDSG_OK;
}
