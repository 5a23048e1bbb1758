// ddsg_mlp.cu -- warm-start network: a GELU MLP trained and evaluated with
// hand-written BF16 tensor-core GEMMs on Blackwell's tcgen05 path (TMA operand
// tiles, FP32 accumulators in tensor memory, fused epilogues).
//
// The network proposes Newton initial guesses for the IRBC step; the paper
// has no network -- the interpolant and the Newton solve decide the result.
//
// Layout: every width is padded to a multiple of 64 with zeros (weights,
// biases, activations); batches are padded to a multiple of 128 rows whose
// inputs and loss gradients are zero. Master weights and Adam moments are
// FP32; GEMM operands are BF16 copies (W and its transpose). Every GEMM
// operand is K-major: training also keeps the transposed BF16 activations and
// output gradients (written by the producing kernels' epilogues), which are the
// K-major operands of the weight-gradient GEMMs (K = the batch).
#include <cuda.h>
#include <cudaTypedefs.h>
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

// Tiles of the tcgen05 GEMM: 128 x 64 output tile (one 64-column TMEM
// accumulator), K in steps of 64 (one 128-byte swizzle atom of BF16), a
// 4-stage TMA ring. Batches are padded to multiples of 128 rows.
constexpr int TBM = 128, TBN = 64, TBK = 64, TNS = 4;
constexpr int GEMM_THREADS = 128;
constexpr int GEMM_SMEM = 1024 + TNS * (TBM + TBN) * TBK * 2 + 256;
constexpr uint32_t kGemmWaitLimit = 1u << 20;   // try_wait polls before a wait gives up (about 4 s)

enum { EPI_STORE = 0, EPI_HIDDEN = 1, EPI_LAST = 2, EPI_GELU_BWD = 3 };

struct Epi {
    float *f;              // FP32 output (STORE, LAST: result; GELU_BWD: dZ)
    int ldf;
    float *z;              // HIDDEN: pre-activation (nullable)
    int ldz;
    __nv_bfloat16 *h;      // HIDDEN: GELU(z) as BF16; GELU_BWD: dZ as BF16
    int ldh;
    __nv_bfloat16 *ht;     // HIDDEN / GELU_BWD: the same values transposed (column-major), nullable
    int ldht;
    const float *bias;     // HIDDEN, LAST
    const float *zp;       // GELU_BWD: pre-activation of the layer below
    int ldzp;
    int64_t zstride;       // STORE with split K: split z writes f + z * zstride
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t ph) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(s_addr(b)), "r"(ph) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t ph) {
    for (uint32_t i = 0; i < kGemmWaitLimit; ++i)
        if (bar_try(b, ph)) return true;
    return false;
}
// TMA: one 2D box (64 K-elements x rows) of a K-major BF16 operand, 128-byte swizzle
__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *m, int k, int row, uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(s_addr(dst)), "l"(m), "r"(k), "r"(row), "r"(s_addr(bar)) : "memory");
}
// Shared-memory matrix descriptor of a K-major tile written by that TMA: rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride offset), 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    return (uint64_t)((s_addr(p) >> 4) & 0x3FFF) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// C[M x N] = A[M x K] * B[N x K]^T, A and B BF16 K-major (TMA maps ta, tb),
// FP32 accumulate in TMEM, one 128 x 64 tile per block. Thread 0 feeds the
// shared-memory ring by TMA, thread 32 issues tcgen05.mma (M = 128, N = 64,
// K = 16 per instruction) and commits each stage back to the producer; the
// four warps then read the accumulator (lane = row) and apply the epilogue.
// Split K: block z covers k in [z*kchunk, min(K, (z+1)*kchunk)) (kchunk a
// multiple of 64) and (STORE only) writes its partial at f + z * zstride. Every
// wait is bounded; a wait that gives up sets *err, the block skips its output,
// waits (bounded) for its copies and MMAs, and frees its TMEM.
template <int EPI>
__global__ void __launch_bounds__(GEMM_THREADS, 1) gemm_tc_kernel(const __grid_constant__ CUtensorMap ta,
                                                                  const __grid_constant__ CUtensorMap tb, int M, int N,
                                                                  int K, int kchunk, Epi e, unsigned *err) {
    extern __shared__ uint8_t gsm_raw[];
    uint8_t *gsm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *As = gsm;
    uint8_t *Bs = gsm + TNS * TBM * TBK * 2;
    uint64_t *full = reinterpret_cast<uint64_t *>(Bs + TNS * TBN * TBK * 2);
    uint64_t *empty = full + TNS;
    uint64_t *done = empty + TNS;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const int nk = ke > kb ? (ke - kb) / TBK : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TNS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tslot)), "r"(TBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    int issued = 0;
    if (threadIdx.x == 0) {
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TNS;
            if (kt >= TNS && !bar_wait(&empty[s], ((kt / TNS) - 1) & 1)) {
                atomicOr(err, 1u);
                break;
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(&full[s])),
                         "r"((TBM + TBN) * TBK * 2) : "memory");
            tma_box(As + s * TBM * TBK * 2, &ta, kb + kt * TBK, m0, &full[s]);
            tma_box(Bs + s * TBN * TBK * 2, &tb, kb + kt * TBK, n0, &full[s]);
            issued = kt + 1;
        }
    } else if (threadIdx.x == 32) {
        // instruction descriptor: F32 accumulate, BF16 A and B, both K-major, N = 64, M = 128
        constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                                   ((uint32_t)(TBM >> 4) << 24);
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TNS;
            if (!bar_wait(&full[s], (kt / TNS) & 1)) {
                atomicOr(err, 2u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t ad = smem_desc(As + s * TBM * TBK * 2), bd = smem_desc(Bs + s * TBN * TBK * 2);
#pragma unroll
            for (int j = 0; j < TBK / 16; ++j) {
                const uint32_t acc = (kt > 0 || j > 0) ? 1u : 0u;
                // the K step of 16 BF16 (32 bytes) advances the descriptors' start address by 2 (16-byte units)
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem), "l"(ad + 2 * j), "l"(bd + 2 * j), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(s_addr(&empty[s])) : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(done))
                     : "memory");
    }
    __syncwarp();
    const bool fin = __all_sync(0xffffffffu, bar_wait(done, 0));
    if (!fin && lane == 0) atomicOr(err, 4u);
    const bool got = fin && nk > 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < TBN; c0 += 16) {
        uint32_t r[16];
        const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                       "=r"(r[15])
                     : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!got || row >= M) continue;
        const int col0 = n0 + c0;             // 16 consecutive columns of this row (N is a multiple of 16)
        if (col0 >= N) continue;
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
        if (EPI == EPI_STORE) {
            float4 *dst = reinterpret_cast<float4 *>(e.f + (int64_t)blockIdx.z * e.zstride + (int64_t)row * e.ldf + col0);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        } else if (EPI == EPI_LAST) {
            const float4 *bs = reinterpret_cast<const float4 *>(e.bias + col0);
            float4 *dst = reinterpret_cast<float4 *>(e.f + (int64_t)row * e.ldf + col0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 b4 = bs[i];
                dst[i] = make_float4(v[4 * i] + b4.x, v[4 * i + 1] + b4.y, v[4 * i + 2] + b4.z, v[4 * i + 3] + b4.w);
            }
        } else {
            // HIDDEN: z = v + bias, out = GELU(z); GELU_BWD: out = dz = v * GELU'(z of the layer below)
            float out[16];
            if (EPI == EPI_HIDDEN) {
                const float4 *bs = reinterpret_cast<const float4 *>(e.bias + col0);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 b4 = bs[i];
                    v[4 * i] += b4.x;
                    v[4 * i + 1] += b4.y;
                    v[4 * i + 2] += b4.z;
                    v[4 * i + 3] += b4.w;
                }
                if (e.z) {
                    float4 *zd = reinterpret_cast<float4 *>(e.z + (int64_t)row * e.ldz + col0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) zd[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) out[i] = gelu_f(v[i]);
            } else {
                const float4 *zp = reinterpret_cast<const float4 *>(e.zp + (int64_t)row * e.ldzp + col0);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 z4 = zp[i];
                    out[4 * i] = v[4 * i] * gelu_grad_f(z4.x);
                    out[4 * i + 1] = v[4 * i + 1] * gelu_grad_f(z4.y);
                    out[4 * i + 2] = v[4 * i + 2] * gelu_grad_f(z4.z);
                    out[4 * i + 3] = v[4 * i + 3] * gelu_grad_f(z4.w);
                }
                float4 *fd = reinterpret_cast<float4 *>(e.f + (int64_t)row * e.ldf + col0);
#pragma unroll
                for (int i = 0; i < 4; ++i) fd[i] = make_float4(out[4 * i], out[4 * i + 1], out[4 * i + 2], out[4 * i + 3]);
            }
            __align__(16) __nv_bfloat162 hb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) hb[i] = __floats2bfloat162_rn(out[2 * i], out[2 * i + 1]);
            uint4 *hd = reinterpret_cast<uint4 *>(e.h + (int64_t)row * e.ldh + col0);
            hd[0] = *reinterpret_cast<const uint4 *>(&hb[0]);
            hd[1] = *reinterpret_cast<const uint4 *>(&hb[4]);
            if (e.ht) {
                // transposed copy: for each column the warp writes 32 consecutive rows
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    e.ht[(int64_t)(col0 + 2 * i) * e.ldht + row] = hb[i].x;
                    e.ht[(int64_t)(col0 + 2 * i + 1) * e.ldht + row] = hb[i].y;
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        // a producer that gave up may have copies in flight: let the issued stages land
        for (int kt = issued > TNS ? issued - TNS : 0; kt < issued; ++kt) bar_wait(&full[kt % TNS], (kt / TNS) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN) : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// TMA map of a K-major BF16 matrix (rows x K, row stride ld elements) with boxes
// of 64 K-elements x box_rows rows; rows past the end read as zero.
bool k_major_map(CUtensorMap *m, const __nv_bfloat16 *base, int64_t rows, int K, int ld, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C = A * B^T on the tensor cores: A (M x K, row stride lda) and B (N x K, row
// stride ldb), both K-major BF16; K a multiple of 64, N a multiple of 64.
template <int EPI>
cudaError_t gemm(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, const Epi &e,
                 unsigned *err, cudaStream_t st, int splits = 1, int kchunk = 0) {
    CUtensorMap ta, tb;
    if (!k_major_map(&ta, A, M, K, lda, TBM) || !k_major_map(&tb, B, N, K, ldb, TBN)) return cudaErrorInvalidValue;
    cudaError_t a = cudaFuncSetAttribute(gemm_tc_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
    if (a != cudaSuccess) return a;
    dim3 grid((unsigned)((N + TBN - 1) / TBN), (unsigned)((M + TBM - 1) / TBM), (unsigned)splits);
    gemm_tc_kernel<EPI><<<grid, GEMM_THREADS, GEMM_SMEM, st>>>(ta, tb, M, N, K, splits > 1 ? kchunk : K, e, err);
    return cudaGetLastError();
}

// Split of the batch dimension (K of the weight-gradient GEMM) so that the
// output tiles times the splits fill the SMs about twice; chunks are multiples of TBK.
void grad_split(int64_t Bp, int Po, int Pi, int sms, int &splits, int &kchunk) {
    const int tiles = ((Po + TBM - 1) / TBM) * ((Pi + TBN - 1) / TBN);
    const int want = std::max(1, (2 * sms + tiles - 1) / tiles);
    const int64_t kmax = std::max<int64_t>(1, Bp / TBK);
    const int s = (int)std::min<int64_t>(want, kmax);
    kchunk = (int)(((Bp + s - 1) / s + TBK - 1) / TBK * TBK);
    splits = (int)((Bp + kchunk - 1) / kchunk);
}

// x (B x n0, FP64 physical) -> (x - shift) * scale as BF16 in B_pad x P0 (zero padding)
// (XT, nullable: the same transposed, P0 x B_pad)
__global__ void mlp_input_kernel(int64_t B, int64_t Bp, int n0, int P0, const double *__restrict__ x,
                                 const double *__restrict__ shift, const double *__restrict__ scale,
                                 __nv_bfloat16 *__restrict__ X, __nv_bfloat16 *__restrict__ XT) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Bp * P0) return;
    const int64_t b = e / P0;
    const int c = (int)(e - b * P0);
    float v = 0.f;
    if (b < B && c < n0) v = (float)((x[b * n0 + c] - shift[c]) * scale[c]);
    X[e] = __float2bfloat16(v);
    if (XT) XT[(int64_t)c * Bp + b] = __float2bfloat16(v);
}

// dY = 2 (Y - T) / (B m) on the normalized targets; loss += sum (Y - T)^2 / (B m)
__global__ void mlp_loss_kernel(int64_t B, int64_t Bp, int m, int PL, const float *__restrict__ Y,
                                const double *__restrict__ y, const double *__restrict__ shift,
                                const double *__restrict__ scale, float *__restrict__ dY,
                                __nv_bfloat16 *__restrict__ dYb, __nv_bfloat16 *__restrict__ dYbT,
                                double *__restrict__ loss) {
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
        dYbT[(int64_t)c * Bp + b] = __float2bfloat16(g);
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

// Split-K sums of one layer in one launch, in z order (deterministic):
// gW[i] = sum_z pw[z*nw + i] for i < nw, then gb[j] = sum_z pb[z*nb + j].
__global__ void splitk_reduce_kernel(int splits, int64_t nw, int64_t nb, const float *__restrict__ pw,
                                     const float *__restrict__ pb, float *__restrict__ gW, float *__restrict__ gb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw + nb) return;
    const bool w = i < nw;
    const int64_t n = w ? nw : nb, j = w ? i : i - nw;
    const float *part = w ? pw : pb;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * n + j];
    (w ? gW : gb)[j] = s;
}

// Parameter tensors of one Adam launch (weights and biases of every layer).
constexpr int kAdamMax = 32;
struct AdamTensor {
    int64_t n, begin;        // elements; first global element of this tensor
    int rows, cols;          // weights: rows x cols (for the transposed BF16 copy)
    float *p, *g, *mo, *ve;
    __nv_bfloat16 *pb, *pbt; // BF16 copy and transposed copy (nullable)
};
struct AdamTable {
    int count;
    int64_t total;
    AdamTensor t[kAdamMax];
};

// Adam over every parameter tensor in one launch (FP32 masters), refreshing the
// BF16 copies and, for weights, the transposed BF16 copies.
__global__ void adam_all_kernel(const AdamTable tab, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t ge = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ge < tab.total;
         ge += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < tab.count && ge >= tab.t[k + 1].begin) ++k;
        const AdamTensor &T = tab.t[k];
        const int64_t e = ge - T.begin;
        const float gr = T.g[e];
        const float m1 = b1 * T.mo[e] + (1.f - b1) * gr;
        const float v1 = b2 * T.ve[e] + (1.f - b2) * gr * gr;
        T.mo[e] = m1;
        T.ve[e] = v1;
        const float np = T.p[e] - lr * (m1 / c1) / (sqrtf(v1 / c2) + eps);
        T.p[e] = np;
        if (T.pb) T.pb[e] = __float2bfloat16(np);
        if (T.pbt) {
            const int r = (int)(e / T.cols), c = (int)(e - (int64_t)r * T.cols);
            T.pbt[(int64_t)c * T.rows + r] = __float2bfloat16(np);
        }
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
inline int64_t pad_rows(int64_t n) { return (n + TBM - 1) & ~(int64_t)(TBM - 1); }   // batch rows: GEMM tile height
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
    unsigned *err = nullptr;      // device word: GEMM waits that gave up (bits by site)
    int sms = 1;                  // SM count of the bound device (split-K sizing)
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
    cudaFree(M->err);
    M->in_shift = M->in_scale = M->out_shift = M->out_scale = nullptr;
    M->loss = nullptr;
    M->err = nullptr;
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
        !alloc((void **)&M->loss, 8) || !alloc((void **)&M->err, 8))
        return set_error(DDSG_ERR_OOM, "mlp: allocation failed");
    if (cudaDeviceGetAttribute(&M->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || M->sms < 1) {
        cudaGetLastError();
        M->sms = 1;
    }
    if (!tensor_map_encoder()) return set_error(DDSG_ERR_CUDA, "mlp: the driver offers no cuTensorMapEncodeTiled");
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
// Training also keeps XT_l (P_l x Bp, the layer inputs transposed) and dZbT
// ping-pong (Pmax x Bp), the K-major operands of the weight-gradient GEMMs.
struct WsView {
    std::vector<__nv_bfloat16 *> X, XT;
    std::vector<float *> Z;
    float *Y;
    float *dZ[2];
    __nv_bfloat16 *dZb[2], *dZbT[2];
    float *split;   // split-K partials of one layer's weight and bias gradients
};

int mlp_ws(mlp *M, int64_t Bp, WsView &v) {
    const int L = M->L;
    int Pmax = 0;
    for (int p : M->P) Pmax = std::max(Pmax, p);
    auto rnd = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t need = 0;
    for (int l = 0; l < L; ++l) need += 2 * rnd((size_t)Bp * M->P[l] * 2);
    for (int l = 0; l + 1 < L; ++l) need += rnd((size_t)Bp * M->P[l + 1] * 4);
    need += rnd((size_t)Bp * M->P[L] * 4);
    need += 2 * rnd((size_t)Bp * Pmax * 4) + 4 * rnd((size_t)Bp * Pmax * 2);
    size_t split_floats = 0;
    for (int l = 0; l < L; ++l) {
        int s = 1, kc = 0;
        grad_split(Bp, M->P[l + 1], M->P[l], M->sms, s, kc);
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
    v.XT.resize(L);
    v.Z.resize(L);
    for (int l = 0; l < L; ++l) v.X[l] = (__nv_bfloat16 *)take((size_t)Bp * M->P[l] * 2);
    for (int l = 0; l < L; ++l) v.XT[l] = (__nv_bfloat16 *)take((size_t)Bp * M->P[l] * 2);
    for (int l = 0; l + 1 < L; ++l) v.Z[l] = (float *)take((size_t)Bp * M->P[l + 1] * 4);
    v.Y = (float *)take((size_t)Bp * M->P[L] * 4);
    for (int i = 0; i < 2; ++i) v.dZ[i] = (float *)take((size_t)Bp * Pmax * 4);
    for (int i = 0; i < 2; ++i) v.dZb[i] = (__nv_bfloat16 *)take((size_t)Bp * Pmax * 2);
    for (int i = 0; i < 2; ++i) v.dZbT[i] = (__nv_bfloat16 *)take((size_t)Bp * Pmax * 2);
    v.split = (float *)take(split_floats * 4);
    return DDSG_OK;
}

// forward pass through all layers; keepZ stores pre-activations for training
cudaError_t mlp_forward(mlp *M, int64_t B, int64_t Bp, const double *x, WsView &v, bool keepZ, cudaStream_t st) {
    const int L = M->L;
    {
        Tracer::Scope ts(&M->tr, 2, st);
        mlp_input_kernel<<<nblk(Bp * M->P[0]), 256, 0, st>>>(B, Bp, M->n[0], M->P[0], x, M->in_shift, M->in_scale,
                                                             v.X[0], keepZ ? v.XT[0] : nullptr);
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
            ep.ht = keepZ ? v.XT[l + 1] : nullptr;
            ep.ldht = (int)Bp;
            e = gemm<EPI_HIDDEN>((int)Bp, M->P[l + 1], M->P[l], v.X[l], M->P[l], M->Wb[l], M->P[l], ep, M->err, st);
        } else {
            ep.f = v.Y;
            ep.ldf = M->P[L];
            e = gemm<EPI_LAST>((int)Bp, M->P[L], M->P[l], v.X[l], M->P[l], M->Wb[l], M->P[l], ep, M->err, st);
        }
    }
    return e;
}

}  // namespace

extern "C" int mlp_create(int nlayers, const int32_t *sizes, const float *params_host, uint64_t seed,
                          mlp_t **out) {
    if (!sizes || !out || nlayers < 1 || nlayers > kAdamMax / 2) return set_error(DDSG_ERR_ARG, "mlp_create: bad argument");
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
        if ((rc = mlp_ws(M, pad_rows(std::min(chunk, B)), v0))) return rc;
    }
    for (int64_t b0 = 0; b0 < B; b0 += chunk) {
        const int64_t nb = std::min(chunk, B - b0);
        const int64_t Bp = pad_rows(nb);
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
    const int64_t Bp = pad_rows(B);
    WsView v;
    if ((rc = mlp_ws(M, Bp, v))) return rc;
    const int L = M->L;
    cudaError_t e = mlp_forward(M, B, Bp, x_dev, v, true, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->loss, 0, 8, st);
    if (e == cudaSuccess) {
        Tracer::Scope ts(&M->tr, 2, st);
        mlp_loss_kernel<<<nblk(Bp * M->P[L]), 256, 0, st>>>(B, Bp, M->n[L], M->P[L], v.Y, y_dev, M->out_shift,
                                                            M->out_scale, v.dZ[0], v.dZb[0], v.dZbT[0], M->loss);
        e = cudaGetLastError();
    }
    // backward: layer l has input width P[l], output width P[l+1]; dZ[cur] holds dL/dZ_l
    int cur = 0;
    for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
        Tracer::Scope ts(&M->tr, 1, st);
        const int Pi = M->P[l], Po = M->P[l + 1];
        // gW = dZ^T (Po x Bp) * X_l (Bp x Pi) = dZbT * XT_l^T, both K-major (K = the
        // batch); the batch is split over blocks, partials summed in split order
        int splits = 1, kchunk = 0;
        grad_split(Bp, Po, Pi, M->sms, splits, kchunk);
        const int64_t nw = (int64_t)Po * Pi;
        float *pw = v.split, *pb = v.split + (int64_t)splits * nw;
        Epi g = {};
        g.f = pw;
        g.ldf = Pi;
        g.zstride = nw;
        e = gemm<EPI_STORE>(Po, Pi, (int)Bp, v.dZbT[cur], (int)Bp, v.XT[l], (int)Bp, g, M->err, st, splits, kchunk);
        if (e == cudaSuccess) {
            colsum_part_kernel<<<dim3((unsigned)((Po + 31) / 32), (unsigned)splits), 256, 0, st>>>(Bp, Po, kchunk,
                                                                                                v.dZ[cur], pb);
            splitk_reduce_kernel<<<nblk(nw + Po), 256, 0, st>>>(splits, nw, Po, pw, pb, M->gW[l], M->gb[l]);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && l > 0) {
            Epi d = {};
            d.f = v.dZ[cur ^ 1];
            d.ldf = Pi;
            d.h = v.dZb[cur ^ 1];
            d.ldh = Pi;
            d.ht = v.dZbT[cur ^ 1];
            d.ldht = (int)Bp;
            d.zp = v.Z[l - 1];
            d.ldzp = Pi;
            // dA = dZ (Bp x Po) * W (Po x Pi) = dZ * (W^T)^T with W^T stored Pi x Po
            e = gemm<EPI_GELU_BWD>((int)Bp, Pi, Po, v.dZb[cur], Po, M->WbT[l], Po, d, M->err, st);
            cur ^= 1;
        }
    }
    // Adam (bias corrections of step t)
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 - pow(0.9, (double)M->step)), c2 = (float)(1.0 - pow(0.999, (double)M->step));
    if (e == cudaSuccess) {
        Tracer::Scope ts(&M->tr, 3, st);
        AdamTable tab = {};
        int64_t off = 0;
        for (int l = 0; l < L; ++l) {
            const int Pi = M->P[l], Po = M->P[l + 1];
            tab.t[tab.count++] = {(int64_t)Pi * Po, off, Po, Pi, M->W[l], M->gW[l], M->mW[l], M->vW[l], M->Wb[l], M->WbT[l]};
            off += (int64_t)Pi * Po;
            tab.t[tab.count++] = {(int64_t)Po, off, 1, Po, M->b[l], M->gb[l], M->mb[l], M->vb[l], nullptr, nullptr};
            off += Po;
        }
        tab.total = off;
        int64_t blocks = nblk(off);
        if (blocks > (int64_t)M->sms * 8) blocks = (int64_t)M->sms * 8;
        adam_all_kernel<<<(unsigned)blocks, 256, 0, st>>>(tab, lr, b1, b2, eps, c1, c2);
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

extern "C" int mlp_check(mlp_t *M) {
    if (!M) return set_error(DDSG_ERR_ARG, "mlp_check: NULL network");
    if (M->device < 0 || !M->err) return DDSG_OK;   // nothing ran yet
    unsigned w = 0;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&w, M->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DDSG_ERR_CUDA, "mlp_check: reading the status word failed");
    }
    if (w) {
        cudaMemset(M->err, 0, 4);
        return set_error(DDSG_ERR_TIMEOUT, "mlp_check: a tensor-core GEMM gave up a bounded wait (its output is incomplete)");
    }
    return DDSG_OK;
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
