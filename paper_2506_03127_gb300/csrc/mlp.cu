// libqp: learned surrogate of rho(t) -- a three-layer MLP with BF16 weights
// and activations and FP32 accumulation, trained and evaluated by the
// kernels of this file (the paper has no counterpart; see include/qp.h).
//
// Network: x (d_in) -> h1 = tanh(x W1 + b1) (width) -> h2 = tanh(h1 W2 + b2)
// (width) -> y = h2 W3 + b3 (d_out).  Loss: mean squared error over the
// batch and the outputs.  Parameters are kept in FP32 (Adam moments too);
// every GEMM reads BF16 copies of its operands (weights re-rounded after each
// update, activations rounded when they are produced) and accumulates in
// FP32 on the tensor cores (mma.sync m16n8k16 BF16 -> FP32).
//
// All GEMMs have the form C[m][n] = sum_k A[m][k] B[n][k] with A and B
// row-major over k ("NT"); K is padded with zeros to a multiple of 32.
//   forward   h = x W  : A = x (batch x K), B = W^T (width x K)
//   backward  dx = dh W^T : A = dh, B = W (in x out, row-major over out)
//   weights   dW = x^T dh : A = x^T (in x batch), B = dh^T (out x batch)
// so each activation is also written transposed (batch contiguous) by the
// kernel that produces it.
//
// Rollout (qp_surrogate_rollout): for up to 32 instances all steps run in
// one launch of a two-block cluster (k_rollout_fused: block 0 keeps W1^T and
// the last L steps of rho in shared memory and runs the feature packing,
// layer 1 and the update; block 1 keeps W2^T and W3^T and runs layers 2 and
// 3; activations cross through distributed shared memory); larger batches
// replay CUDA graphs of the per-step kernels.  Both round at the same points
// and add the k-steps in the same order.
//
// Tensor-core form: warp-level mma.sync fragments.  These GEMMs are small
// (at most a few thousand rows by 258 x 256 in training, 16 rows per
// rollout step); tcgen05.mma issues 64- or 128-row tiles through tensor
// memory, which a 16-row step would fill to a quarter while adding a
// tensor-memory round trip to a step whose cost is latency.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qp.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 32;   // block tile
constexpr int kGemmThreads = 128;          // 4 warps, 2 x 2, 32 x 32 each
constexpr int SPAD = 8;                    // smem row padding (bf16) against bank conflicts

__host__ __device__ inline int pad32(int x) { return (x + 31) & ~31; }

enum Epi { EPI_TANH = 0, EPI_LINEAR = 1, EPI_DTANH = 2, EPI_STORE = 3 };

struct EpiArgs {
    const float *bias;        // [N] (TANH, LINEAR)
    float *out_f32;           // [M x ldo] FP32 result (TANH: h, LINEAR: y, STORE: C)
    int ldo;
    __nv_bfloat16 *out_bf;    // [M x ldb] BF16 copy, row-major (TANH, DTANH)
    int ldb;
    __nv_bfloat16 *out_bfT;   // [N x ldt] BF16 copy, transposed (TANH, DTANH)
    int ldt;
    const float *h;           // DTANH: tanh output of the layer, [M x ldh]
    int ldh;
    float *colsum;            // DTANH: += column sums of the result (bias gradient)
};

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldmatrix_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldmatrix_x2(unsigned &r0, unsigned &r1, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float *c, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C = A B^T over K (multiple of 32); rows of A beyond M and rows of B beyond
// N read as zero; the epilogue is applied to the valid M x N part.
template <int EPI>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_nt(const __nv_bfloat16 *__restrict__ A, int lda,
                                                          const __nv_bfloat16 *__restrict__ B, int ldb, int M, int N,
                                                          int K, EpiArgs ep) {
    __shared__ __align__(16) __nv_bfloat16 sA[BM][BK + SPAD];
    __shared__ __align__(16) __nv_bfloat16 sB[BN][BK + SPAD];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    for (int k0 = 0; k0 < K; k0 += BK) {
        // 64 rows x 32 bf16 = 256 chunks of 16 B per operand, 2 per thread
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int chunk = threadIdx.x + c * kGemmThreads;
            const int r = chunk >> 2, kc = (chunk & 3) * 8;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + r < M) va = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + k0 + kc);
            if (n0 + r < N) vb = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * ldb + k0 + kc);
            *reinterpret_cast<uint4 *>(&sA[r][kc]) = va;
            *reinterpret_cast<uint4 *>(&sB[r][kc]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm + i * 16 + (lane & 15);
                const int col = kk + (lane >> 4) * 8;
                ldmatrix_x4(a[i][0], a[i][1], a[i][2], a[i][3], &sA[row][col]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int row = wn + j * 8 + (lane & 7);
                const int col = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x2(b[j][0], b[j][1], &sB[row][col]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i][0], a[i][1], a[i][2], a[i][3], b[j][0], b[j][1]);
        }
        __syncthreads();
    }
    // epilogue: acc[i][j][r] is C[m][n] with m = wm + 16 i + g (+8 for r >= 2),
    // n = wn + 8 j + 2 t (+1 for odd r), g = lane / 4, t = lane % 4
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * t + (r & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][r];
                if constexpr (EPI == EPI_TANH) {
                    v = tanhf(v + ep.bias[n]);
                    ep.out_f32[(size_t)m * ep.ldo + n] = v;
                    const __nv_bfloat16 vb = __float2bfloat16_rn(v);
                    ep.out_bf[(size_t)m * ep.ldb + n] = vb;
                    ep.out_bfT[(size_t)n * ep.ldt + m] = vb;
                } else if constexpr (EPI == EPI_LINEAR) {
                    ep.out_f32[(size_t)m * ep.ldo + n] = v + ep.bias[n];
                } else if constexpr (EPI == EPI_DTANH) {
                    const float hv = ep.h[(size_t)m * ep.ldh + n];
                    v *= 1.f - hv * hv;
                    const __nv_bfloat16 vb = __float2bfloat16_rn(v);
                    ep.out_bf[(size_t)m * ep.ldb + n] = vb;
                    ep.out_bfT[(size_t)n * ep.ldt + m] = vb;
                    atomicAdd(&ep.colsum[n], v);
                } else {
                    ep.out_f32[(size_t)m * ep.ldo + n] = v;
                }
            }
}

// x (FP32, batch x d_in) -> BF16 row-major (ld = pad32(d_in)) and transposed
// (ld = pad32(batch)); pads stay zero (written once at create).
__global__ void k_pack_input(const float *x, int batch, int d_in, __nv_bfloat16 *xb, int ldx, __nv_bfloat16 *xT,
                             int ldt) {
    const long long total = (long long)batch * d_in;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i / d_in), k = (int)(i % d_in);
        const __nv_bfloat16 v = __float2bfloat16_rn(x[i]);
        xb[(size_t)m * ldx + k] = v;
        xT[(size_t)k * ldt + m] = v;
    }
}

// dy = 2 (y - target) / (batch d_out) -> BF16 (row-major, ld 32, and
// transposed); db3 = column sums; loss partial sums.
__global__ void k_loss_grad(const float *y, const float *tgt, int batch, int d_out, __nv_bfloat16 *dyb, int lddy,
                            __nv_bfloat16 *dyT, int ldt, float *db3, double *loss) {
    __shared__ double s_l[256];
    double l = 0.0;
    const float scale = 2.f / (float)(batch * d_out);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch * d_out; i += gridDim.x * blockDim.x) {
        const int m = i / d_out, n = i % d_out;
        const float e = y[i] - tgt[i];
        l += (double)e * e;
        const float d = scale * e;
        const __nv_bfloat16 db = __float2bfloat16_rn(d);
        dyb[(size_t)m * lddy + n] = db;
        dyT[(size_t)n * ldt + m] = db;
        atomicAdd(&db3[n], d);
    }
    s_l[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s_l[threadIdx.x] += s_l[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, s_l[0] / (double)(batch * d_out));
}

// Adam on FP32 parameters, then the BF16 copies the GEMMs read: W (row-major
// in x out, ld pad32(out)) and W^T (out x in, ld pad32(in)).
struct ParamBlock {
    float *w, *g, *m, *v;        // [rows x cols] FP32 (row-major rows x cols)
    int rows, cols;              // in x out for weights, 1 x out for biases
    __nv_bfloat16 *wb, *wbT;     // BF16 copies (weights only)
    int ldb, ldt;
};

__global__ void k_adam(ParamBlock p, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    const int n = p.rows * p.cols;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = p.g[i];
        const float m = b1 * p.m[i] + (1.f - b1) * g;
        const float v = b2 * p.v[i] + (1.f - b2) * g * g;
        p.m[i] = m;
        p.v[i] = v;
        const float w = p.w[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        p.w[i] = w;
        if (p.wb) {
            const int r = i / p.cols, c = i % p.cols;
            const __nv_bfloat16 wb = __float2bfloat16_rn(w);
            p.wb[(size_t)r * p.ldb + c] = wb;
            p.wbT[(size_t)c * p.ldt + r] = wb;
        }
    }
}

__global__ void k_round_weights(ParamBlock p) {
    const int n = p.rows * p.cols;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = i / p.cols, c = i % p.cols;
        const __nv_bfloat16 wb = __float2bfloat16_rn(p.w[i]);
        p.wb[(size_t)r * p.ldb + c] = wb;
        p.wbT[(size_t)c * p.ldt + r] = wb;
    }
}

// ---------------------------------------------------------------- surrogate data path

// Windows of rho trajectories: for instance i and target time t (t_begin <=
// t < t_end), features = the 8 reals (Re, Im of rho_00, rho_01, rho_10,
// rho_11) of rho(t-L) .. rho(t-1), then the instance's n_par parameters;
// target = (rho(t) - rho(t-1)) * out_scale.  rho: [T][n_inst][4] double2.
__global__ void k_windows(const double2 *rho, int n_inst, int L, const float *par, int n_par, int t_begin, int t_end,
                          int inst0, int ninst_used, float out_scale, float *x, float *tgt) {
    const int per = t_end - t_begin;
    const int d_in = 8 * L + n_par;
    const long long total = (long long)ninst_used * per * d_in;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(idx % d_in);
        const long long row = idx / d_in;
        const int ii = (int)(row / per), t = t_begin + (int)(row % per);
        const int inst = inst0 + ii;
        float v;
        if (f < 8 * L) {
            const int s = t - L + f / 8, e = (f % 8) / 2;
            const double2 z = rho[((size_t)s * n_inst + inst) * 4 + e];
            v = (float)((f & 1) ? z.y : z.x);
        } else {
            v = par[(size_t)inst * n_par + (f - 8 * L)];
        }
        x[idx] = v;
        if (f < 8) {
            const double2 a = rho[((size_t)t * n_inst + inst) * 4 + f / 2];
            const double2 b = rho[((size_t)(t - 1) * n_inst + inst) * 4 + f / 2];
            tgt[row * 8 + f] = (float)(((f & 1) ? (a.y - b.y) : (a.x - b.x)) * out_scale);
        }
    }
}

// Rollout input: features of step t (= *tstep) from the history hist
// [n][T][8] (FP32): the last L values of rho and the bath parameters.  The
// step index lives on the device so that a captured graph of steps can be
// replayed.  They are rounded to BF16 straight into row i of the first
// layer's input (ld = ldx; pads stay zero): the rollout needs no FP32 copy
// and no transposed one (that is for the weight gradients of training).
__global__ void k_rollout_pack(const float *hist, int n, int T, int L, const float *par, int n_par,
                               const int *tstep, __nv_bfloat16 *xb, int ldx) {
    const int t = *tstep;
    const int d_in = 8 * L + n_par;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * d_in; idx += gridDim.x * blockDim.x) {
        const int i = idx / d_in, f = idx % d_in;
        const float v = f < 8 * L ? hist[((size_t)i * T + (t - L + f / 8)) * 8 + (f % 8)] : par[(size_t)i * n_par + f - 8 * L];
        xb[(size_t)i * ldx + f] = __float2bfloat16_rn(v);
    }
}

// rho(t) = rho(t-1) + y / out_scale with the increment made traceless (the
// trace changes only through the filter, negligibly over a rollout), then
// projected onto Hermitian matrices (rho_10 = conj rho_01 from their mean,
// real diagonal) and onto positive semidefinite ones of the same trace.
// The last block to finish advances the step index (every block has read
// it by then).
__global__ void k_rollout_update(float *hist, int n, int T, int *tstep, unsigned *done, const float *y,
                                 float out_scale) {
    const int t = *tstep;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        *done = 0;
        *tstep = t + 1;
    }
    if (i >= n) return;
    const float *prev = hist + ((size_t)i * T + (t - 1)) * 8;
    float d[8];
    for (int k = 0; k < 8; ++k) d[k] = y[i * 8 + k] / out_scale;
    const float tr = 0.5f * (d[0] + d[6]);
    d[0] -= tr;
    d[6] -= tr;
    float r[8];
    for (int k = 0; k < 8; ++k) r[k] = prev[k] + d[k];
    const float re = 0.5f * (r[2] + r[4]), im = 0.5f * (r[3] - r[5]);
    r[2] = re;
    r[3] = im;
    r[4] = re;
    r[5] = -im;
    r[1] = 0.f;
    r[7] = 0.f;
    // positive semidefinite: with c = tr/2, z = (rho_00 - rho_11)/2, b =
    // rho_01 the eigenvalues are c +- sqrt(z^2 + |b|^2); a radius above c is
    // scaled back to c (the nearest such state of the same trace)
    const float c = 0.5f * (r[0] + r[6]), z = 0.5f * (r[0] - r[6]);
    const float rad = sqrtf(z * z + r[2] * r[2] + r[3] * r[3]);
    if (c > 0.f && rad > c) {
        const float f = c / rad;
        r[0] = c + f * z;
        r[6] = c - f * z;
        r[2] *= f;
        r[3] *= f;
        r[4] = r[2];
        r[5] = -r[3];
    }
    float *out = hist + ((size_t)i * T + t) * 8;
    for (int k = 0; k < 8; ++k) out[k] = r[k];
}

// The whole rollout in one launch of a two-block cluster (the batch is one
// or two m16 tiles).  Block 0 keeps the first layer's weights W1^T in
// shared memory and the last L steps of rho in a ring (when it fits): per
// step it packs the features (BF16), runs layer 1 and writes h1 into block
// 1's shared memory; block 1 keeps W2^T and W3^T, runs layers 2 and 3 and
// writes y back into block 0, which applies the update of k_rollout_update.
// Two cluster barriers per step; no launch, no global round trip.  The
// layers are m16n8k16 BF16 MMAs with FP32 accumulation over the k-steps in
// ascending order and the epilogues of k_gemm_nt (tanh and BF16 rounding of
// the next layer's input; bias): the same rounding points and summation
// order as the kernel-by-kernel rollout.  Shared memory, the same layout in
// both blocks: weights (block 0: W1^T [width][K1 + 8]; block 1: W2^T
// [width][Kw + 8] then W3^T [8][Kw + 8]), features [16 MT][K1 + 8], h1, h2
// [16 MT][Kw + 8] (BF16), y [16 MT][8] and the ring [n][L][8] (FP32); rows
// past n and columns past the layer widths stay zero.
struct RollArgs {
    float *hist;
    const float *par;
    const __nv_bfloat16 *w1t, *w2t, *w3t;   // W^T, rows of K1, Kw, Kw
    const float *b1, *b2, *b3;
    int n, T, L, n_par, d_in, width, K1, Kw, t_from, t_to, ring;
    float out_scale;
};
constexpr int kRollThreads = 256;
constexpr int kRollNT = 4;   // n-tiles of a warp per pass (A fragments shared)

__host__ __device__ inline size_t roll_weight_elems(int width, int K1, int Kw) {
    const size_t w1 = (size_t)width * (K1 + 8), w23 = (size_t)(width + 8) * (Kw + 8);
    return w1 > w23 ? w1 : w23;
}
inline size_t roll_smem_bytes(int MT, int width, int K1, int Kw, int n, int L, bool ring) {
    return roll_weight_elems(width, K1, Kw) * 2 + (size_t)16 * MT * (K1 + 8) * 2 +
           (size_t)2 * 16 * MT * (Kw + 8) * 2 + (size_t)16 * MT * 8 * 4 + (ring ? (size_t)n * L * 8 * 4 : 0);
}

// NTW m16n8 tiles of C = A B^T over K (ascending k-steps of 16): A [16 MT
// rows][lda] and B = W^T [rows][ldb] in shared memory; tile j covers
// columns n0 + j * nstride (tiles at or past nmax are computed from row 0
// and not used); acc[j][mt][r] as in k_gemm_nt's epilogue
template <int MT, int NTW>
__device__ __forceinline__ void roll_tiles(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int n0,
                                           int nstride, int nmax, int K, float (*acc)[MT][4]) {
    const int lane = threadIdx.x & 31;
    const __nv_bfloat16 *brow[NTW];
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
        const int nj = n0 + j * nstride < nmax ? n0 + j * nstride : 0;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[j][mt][r] = 0.f;
        brow[j] = B + (size_t)(nj + (lane & 7)) * ldb + ((lane >> 3) & 1) * 8;
    }
#pragma unroll 2
    for (int kk = 0; kk < K; kk += 16) {
        unsigned b0[NTW], b1[NTW];
#pragma unroll
        for (int j = 0; j < NTW; ++j) ldmatrix_x2(b0[j], b1[j], brow[j] + kk);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            unsigned a0, a1, a2, a3;
            ldmatrix_x4(a0, a1, a2, a3, A + (size_t)(mt * 16 + (lane & 15)) * lda + kk + (lane >> 4) * 8);
#pragma unroll
            for (int j = 0; j < NTW; ++j) mma_bf16(acc[j][mt], a0, a1, a2, a3, b0[j], b1[j]);
        }
    }
}

// rows of a row-major BF16 matrix (rows x K, K a multiple of 8) into shared
// memory rows of ld elements, 16-byte chunks
__device__ __forceinline__ void roll_copy_rows(__nv_bfloat16 *dst, int ld, const __nv_bfloat16 *src, int rows, int K) {
    for (int i = threadIdx.x; i < rows * (K / 8); i += kRollThreads) {
        const int r = i / (K / 8), c = (i % (K / 8)) * 8;
        *reinterpret_cast<uint4 *>(dst + (size_t)r * ld + c) = *reinterpret_cast<const uint4 *>(src + (size_t)r * K + c);
    }
}

template <int MT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kRollThreads) k_rollout_fused(RollArgs a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    extern __shared__ __align__(16) unsigned char s_roll[];
    const int l1 = a.K1 + 8, lw = a.Kw + 8;
    __nv_bfloat16 *sW = reinterpret_cast<__nv_bfloat16 *>(s_roll);
    __nv_bfloat16 *sX = sW + roll_weight_elems(a.width, a.K1, a.Kw);
    __nv_bfloat16 *sH1 = sX + (size_t)16 * MT * l1;
    __nv_bfloat16 *sH2 = sH1 + (size_t)16 * MT * lw;
    float *sY = reinterpret_cast<float *>(sH2 + (size_t)16 * MT * lw);
    float *sRing = sY + 16 * MT * 8;   // [n][L][8]: step s at slot s % L
    __nv_bfloat16 *peerH1 = cluster.map_shared_rank(sH1, 1);   // block 0 writes h1 there
    float *peerY = cluster.map_shared_rank(sY, 0);             // block 1 writes y there
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kRollThreads / 32;
    const int g = lane >> 2, tq = lane & 3;
    if (rank == 0) {
        roll_copy_rows(sW, l1, a.w1t, a.width, a.K1);
        for (int i = threadIdx.x; i < 16 * MT * l1; i += kRollThreads) sX[i] = __float2bfloat16_rn(0.f);
        if (a.ring)
            for (int idx = threadIdx.x; idx < a.n * a.L * 8; idx += kRollThreads) {
                const int i = idx / (a.L * 8), s = a.t_from - a.L + (idx / 8) % a.L, k = idx % 8;
                sRing[((size_t)i * a.L + s % a.L) * 8 + k] = a.hist[((size_t)i * a.T + s) * 8 + k];
            }
    } else {
        roll_copy_rows(sW, lw, a.w2t, a.width, a.Kw);
        roll_copy_rows(sW + (size_t)a.width * lw, lw, a.w3t, 8, a.Kw);
        for (int i = threadIdx.x; i < 2 * 16 * MT * lw; i += kRollThreads) sH1[i] = __float2bfloat16_rn(0.f);
    }
    cluster.sync();
    for (int t = a.t_from; t < a.t_to; ++t) {
        if (rank == 0) {
            // features of step t: the last L values of rho, then the parameters
            const int s0 = (t - a.L) % a.L;
            for (int idx = threadIdx.x; idx < a.n * a.d_in; idx += kRollThreads) {
                const int i = idx / a.d_in, f = idx - i * a.d_in;
                float v;
                if (f >= 8 * a.L) {
                    v = a.par[(size_t)i * a.n_par + f - 8 * a.L];
                } else if (a.ring) {
                    int slot = s0 + (f >> 3);
                    slot = slot >= a.L ? slot - a.L : slot;
                    v = sRing[((size_t)i * a.L + slot) * 8 + (f & 7)];
                } else {
                    v = a.hist[((size_t)i * a.T + (t - a.L + (f >> 3))) * 8 + (f & 7)];
                }
                sX[(size_t)i * l1 + f] = __float2bfloat16_rn(v);
            }
            __syncthreads();
            // layer 1: a warp's n-tiles nb + j * 64; h1 = tanh(acc + b1), BF16, into block 1
            for (int nb = warp * 8; nb < a.width; nb += nw * 8 * kRollNT) {
                float acc[kRollNT][MT][4];
                roll_tiles<MT, kRollNT>(sX, l1, sW, l1, nb, nw * 8, a.width, a.K1, acc);
#pragma unroll
                for (int j = 0; j < kRollNT; ++j)
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int m = mt * 16 + g + (r >= 2 ? 8 : 0);
                            const int n = nb + j * nw * 8 + 2 * tq + (r & 1);
                            if (m < a.n && n < a.width)
                                peerH1[(size_t)m * lw + n] = __float2bfloat16_rn(tanhf(acc[j][mt][r] + a.b1[n]));
                        }
            }
        }
        cluster.sync();   // h1 in block 1
        if (rank == 1) {
            // layer 2: h2 = tanh(h1 W2 + b2), BF16
            for (int nb = warp * 8; nb < a.width; nb += nw * 8 * kRollNT) {
                float acc[kRollNT][MT][4];
                roll_tiles<MT, kRollNT>(sH1, lw, sW, lw, nb, nw * 8, a.width, a.Kw, acc);
#pragma unroll
                for (int j = 0; j < kRollNT; ++j)
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int m = mt * 16 + g + (r >= 2 ? 8 : 0);
                            const int n = nb + j * nw * 8 + 2 * tq + (r & 1);
                            if (m < a.n && n < a.width)
                                sH2[(size_t)m * lw + n] = __float2bfloat16_rn(tanhf(acc[j][mt][r] + a.b2[n]));
                        }
            }
            __syncthreads();
            // layer 3: y = h2 W3 + b3 (8 outputs: one n-tile), warp 0, into block 0
            if (warp == 0) {
                float acc[1][MT][4];
                roll_tiles<MT, 1>(sH2, lw, sW + (size_t)a.width * lw, lw, 0, 8, 8, a.Kw, acc);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int m = mt * 16 + g + (r >= 2 ? 8 : 0), n = 2 * tq + (r & 1);
                        if (m < a.n) peerY[m * 8 + n] = acc[0][mt][r] + a.b3[n];
                    }
            }
        }
        cluster.sync();   // y in block 0
        if (rank == 0) {
            // the update of k_rollout_update for instance i
            for (int i = threadIdx.x; i < a.n; i += kRollThreads) {
                const float *prev = a.ring ? sRing + ((size_t)i * a.L + (t - 1) % a.L) * 8
                                           : a.hist + ((size_t)i * a.T + (t - 1)) * 8;
                float d[8];
                for (int k = 0; k < 8; ++k) d[k] = sY[i * 8 + k] / a.out_scale;
                const float tr = 0.5f * (d[0] + d[6]);
                d[0] -= tr;
                d[6] -= tr;
                float r[8];
                for (int k = 0; k < 8; ++k) r[k] = prev[k] + d[k];
                const float re = 0.5f * (r[2] + r[4]), im = 0.5f * (r[3] - r[5]);
                r[2] = re;
                r[3] = im;
                r[4] = re;
                r[5] = -im;
                r[1] = 0.f;
                r[7] = 0.f;
                const float c = 0.5f * (r[0] + r[6]), z = 0.5f * (r[0] - r[6]);
                const float rad = sqrtf(z * z + r[2] * r[2] + r[3] * r[3]);
                if (c > 0.f && rad > c) {
                    const float f = c / rad;
                    r[0] = c + f * z;
                    r[6] = c - f * z;
                    r[2] *= f;
                    r[3] *= f;
                    r[4] = r[2];
                    r[5] = -r[3];
                }
                float *out = a.hist + ((size_t)i * a.T + t) * 8;
                float *slot = sRing + ((size_t)i * a.L + t % a.L) * 8;
                for (int k = 0; k < 8; ++k) {
                    out[k] = r[k];
                    if (a.ring) slot[k] = r[k];
                }
            }
            __syncthreads();
        }
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct qp_mlp {
    int d_in, width, d_out, max_batch;
    int K1, Kw, Ko, Bp;          // padded: d_in, width, d_out (to 32), batch (to 32)
    char *ws = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    // FP32 parameters, gradients, Adam moments: one contiguous block each
    float *par, *grad, *mom, *vel;
    long long npar;
    // views
    float *W[3], *b[3], *gW[3], *gb[3];
    __nv_bfloat16 *Wb[3], *WbT[3];   // W row-major (in x pad(out)), W^T (out x pad(in))
    // activations
    __nv_bfloat16 *xb, *xT, *h1b, *h1T, *h2b, *h2T, *dyb, *dyT, *dh2b, *dh2T, *dh1b, *dh1T;
    float *h1, *h2, *y;
    double *loss;
    int *tstep;                   // rollout step index and block counter (device)
    unsigned *tdone;
    // rollout graph: steps captured once, replayed (key: arguments it bakes in)
    cudaGraphExec_t roll_exec = nullptr, roll_exec_rem = nullptr;
    int roll_steps = 0, roll_rem = 0;
    const void *roll_key[4] = {nullptr, nullptr, nullptr, nullptr};
    int roll_dims[6] = {0, 0, 0, 0, 0, 0};
    float roll_scale = 0.f;
    int roll_mode = QP_ROLLOUT_AUTO;   // fused one-block kernel or the graph of step kernels
    long long step = 0;
    int last_batch = -1;          // batch of the last backward pass (transposed pads)
    std::string err;
};

namespace {

bool mlp_dims_ok(int d_in, int width, int d_out, int max_batch) {
    return d_in >= 1 && d_in <= 4096 && width >= 1 && width <= 4096 && d_out >= 1 && d_out <= 4096 &&
           max_batch >= 1 && max_batch <= (1 << 20);
}

size_t mlp_layout(qp_mlp *m, int d_in, int width, int d_out, int max_batch, char *base) {
    const int K1 = pad32(d_in), Kw = pad32(width), Ko = pad32(d_out), Bp = pad32(max_batch);
    const long long npar = (long long)d_in * width + width + (long long)width * width + width +
                           (long long)width * d_out + d_out;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align256(off + b); return base ? base + o : nullptr; };
    if (m) {
        m->d_in = d_in;
        m->width = width;
        m->d_out = d_out;
        m->max_batch = max_batch;
        m->K1 = K1;
        m->Kw = Kw;
        m->Ko = Ko;
        m->Bp = Bp;
        m->npar = npar;
    }
    char *par = take(npar * 4), *grad = take(npar * 4), *mom = take(npar * 4), *vel = take(npar * 4);
    char *wb[3], *wbT[3];
    const int ins[3] = {d_in, width, width}, outs[3] = {width, width, d_out};
    const int ldin[3] = {K1, Kw, Kw}, ldout[3] = {Kw, Kw, Ko};
    for (int l = 0; l < 3; ++l) {
        wb[l] = take((size_t)ins[l] * ldout[l] * 2);     // W: in x pad(out)
        wbT[l] = take((size_t)outs[l] * ldin[l] * 2);    // W^T: out x pad(in)
    }
    char *xb = take((size_t)max_batch * K1 * 2), *xT = take((size_t)K1 * Bp * 2);
    char *h1b = take((size_t)max_batch * Kw * 2), *h1T = take((size_t)Kw * Bp * 2);
    char *h2b = take((size_t)max_batch * Kw * 2), *h2T = take((size_t)Kw * Bp * 2);
    char *dyb = take((size_t)max_batch * Ko * 2), *dyT = take((size_t)Ko * Bp * 2);
    char *dh2b = take((size_t)max_batch * Kw * 2), *dh2T = take((size_t)Kw * Bp * 2);
    char *dh1b = take((size_t)max_batch * Kw * 2), *dh1T = take((size_t)Kw * Bp * 2);
    char *h1 = take((size_t)max_batch * width * 4), *h2 = take((size_t)max_batch * width * 4);
    char *y = take((size_t)max_batch * d_out * 4), *loss = take(8);
    char *tstep = take(16);
    if (m && base) {
        m->par = (float *)par;
        m->grad = (float *)grad;
        m->mom = (float *)mom;
        m->vel = (float *)vel;
        long long o = 0;
        for (int l = 0; l < 3; ++l) {
            m->W[l] = m->par + o;
            m->gW[l] = m->grad + o;
            o += (long long)ins[l] * outs[l];
            m->b[l] = m->par + o;
            m->gb[l] = m->grad + o;
            o += outs[l];
            m->Wb[l] = (__nv_bfloat16 *)wb[l];
            m->WbT[l] = (__nv_bfloat16 *)wbT[l];
        }
        m->xb = (__nv_bfloat16 *)xb;
        m->xT = (__nv_bfloat16 *)xT;
        m->h1b = (__nv_bfloat16 *)h1b;
        m->h1T = (__nv_bfloat16 *)h1T;
        m->h2b = (__nv_bfloat16 *)h2b;
        m->h2T = (__nv_bfloat16 *)h2T;
        m->dyb = (__nv_bfloat16 *)dyb;
        m->dyT = (__nv_bfloat16 *)dyT;
        m->dh2b = (__nv_bfloat16 *)dh2b;
        m->dh2T = (__nv_bfloat16 *)dh2T;
        m->dh1b = (__nv_bfloat16 *)dh1b;
        m->dh1T = (__nv_bfloat16 *)dh1T;
        m->tstep = (int *)tstep;
        m->tdone = (unsigned *)(tstep + 8);
        m->h1 = (float *)h1;
        m->h2 = (float *)h2;
        m->y = (float *)y;
        m->loss = (double *)loss;
    }
    return off;
}

ParamBlock weight_block(qp_mlp *m, int l, bool with_bf) {
    const int ins[3] = {m->d_in, m->width, m->width}, outs[3] = {m->width, m->width, m->d_out};
    const int ldin[3] = {m->K1, m->Kw, m->Kw}, ldout[3] = {m->Kw, m->Kw, m->Ko};
    const long long off = m->W[l] - m->par;
    ParamBlock p;
    p.w = m->W[l];
    p.g = m->gW[l];
    p.m = m->mom + off;
    p.v = m->vel + off;
    p.rows = ins[l];
    p.cols = outs[l];
    p.wb = with_bf ? m->Wb[l] : nullptr;
    p.wbT = with_bf ? m->WbT[l] : nullptr;
    p.ldb = ldout[l];
    p.ldt = ldin[l];
    return p;
}

ParamBlock bias_block(qp_mlp *m, int l) {
    const int outs[3] = {m->width, m->width, m->d_out};
    const long long off = m->b[l] - m->par;
    ParamBlock p{};
    p.w = m->b[l];
    p.g = m->gb[l];
    p.m = m->mom + off;
    p.v = m->vel + off;
    p.rows = 1;
    p.cols = outs[l];
    return p;
}

template <int EPI>
cudaError_t gemm(qp_mlp *m, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K,
                 const EpiArgs &ep) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm_nt<EPI><<<grid, kGemmThreads, 0, m->stream>>>(A, lda, B, ldb, M, N, K, ep);
    return cudaGetLastError();
}

// The three layers on the packed input m->xb.
cudaError_t forward_layers(qp_mlp *m, int batch) {
    EpiArgs e1{};
    e1.bias = m->b[0];
    e1.out_f32 = m->h1;
    e1.ldo = m->width;
    e1.out_bf = m->h1b;
    e1.ldb = m->Kw;
    e1.out_bfT = m->h1T;
    e1.ldt = m->Bp;
    cudaError_t e = gemm<EPI_TANH>(m, m->xb, m->K1, m->WbT[0], m->K1, batch, m->width, m->K1, e1);
    if (e != cudaSuccess) return e;
    EpiArgs e2 = e1;
    e2.bias = m->b[1];
    e2.out_f32 = m->h2;
    e2.out_bf = m->h2b;
    e2.out_bfT = m->h2T;
    e = gemm<EPI_TANH>(m, m->h1b, m->Kw, m->WbT[1], m->Kw, batch, m->width, m->Kw, e2);
    if (e != cudaSuccess) return e;
    EpiArgs e3{};
    e3.bias = m->b[2];
    e3.out_f32 = m->y;
    e3.ldo = m->d_out;
    return gemm<EPI_LINEAR>(m, m->h2b, m->Kw, m->WbT[2], m->Kw, batch, m->d_out, m->Kw, e3);
}

cudaError_t forward(qp_mlp *m, const float *d_x, int batch) {
    k_pack_input<<<256, 256, 0, m->stream>>>(d_x, batch, m->d_in, m->xb, m->K1, m->xT, m->Bp);
    return forward_layers(m, batch);
}

// The weight-gradient GEMMs contract over the batch padded to 32: the
// transposed activation buffers must be zero beyond the current batch.
cudaError_t clear_transposed(qp_mlp *m, int batch) {
    if (batch == m->last_batch) return cudaSuccess;
    m->last_batch = batch;
    const size_t Bp2 = (size_t)m->Bp * 2;
    cudaError_t e = cudaMemsetAsync(m->xT, 0, m->K1 * Bp2, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->h1T, 0, m->Kw * Bp2, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->h2T, 0, m->Kw * Bp2, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->dyT, 0, m->Ko * Bp2, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->dh2T, 0, m->Kw * Bp2, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->dh1T, 0, m->Kw * Bp2, m->stream);
    return e;
}

cudaError_t backward(qp_mlp *m, const float *d_t, int batch) {
    const int Kb = pad32(batch);
    cudaError_t e = cudaMemsetAsync(m->grad, 0, m->npar * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
    if (e != cudaSuccess) return e;
    k_loss_grad<<<64, 256, 0, m->stream>>>(m->y, d_t, batch, m->d_out, m->dyb, m->Ko, m->dyT, m->Bp, m->gb[2], m->loss);
    EpiArgs st{};
    // dW3 = h2^T dy (width x d_out), contraction over the batch
    st.out_f32 = m->gW[2];
    st.ldo = m->d_out;
    e = gemm<EPI_STORE>(m, m->h2T, m->Bp, m->dyT, m->Bp, m->width, m->d_out, Kb, st);
    if (e != cudaSuccess) return e;
    // dh2 = (dy W3^T) * (1 - h2^2); W3 row-major (width x pad(d_out)) is B
    EpiArgs d2{};
    d2.out_bf = m->dh2b;
    d2.ldb = m->Kw;
    d2.out_bfT = m->dh2T;
    d2.ldt = m->Bp;
    d2.h = m->h2;
    d2.ldh = m->width;
    d2.colsum = m->gb[1];
    e = gemm<EPI_DTANH>(m, m->dyb, m->Ko, m->Wb[2], m->Ko, batch, m->width, m->Ko, d2);
    if (e != cudaSuccess) return e;
    // dW2 = h1^T dh2
    st.out_f32 = m->gW[1];
    st.ldo = m->width;
    e = gemm<EPI_STORE>(m, m->h1T, m->Bp, m->dh2T, m->Bp, m->width, m->width, Kb, st);
    if (e != cudaSuccess) return e;
    // dh1 = (dh2 W2^T) * (1 - h1^2)
    EpiArgs d1 = d2;
    d1.out_bf = m->dh1b;
    d1.out_bfT = m->dh1T;
    d1.h = m->h1;
    d1.colsum = m->gb[0];
    e = gemm<EPI_DTANH>(m, m->dh2b, m->Kw, m->Wb[1], m->Kw, batch, m->width, m->Kw, d1);
    if (e != cudaSuccess) return e;
    // dW1 = x^T dh1
    st.out_f32 = m->gW[0];
    st.ldo = m->width;
    return gemm<EPI_STORE>(m, m->xT, m->Bp, m->dh1T, m->Bp, m->d_in, m->width, Kb, st);
}

qp_status mfail(qp_mlp *m, qp_status s, const std::string &msg) {
    if (m) m->err = msg;
    return s;
}

}  // namespace

extern "C" {

qp_status qp_mlp_workspace_size(int d_in, int width, int d_out, int max_batch, size_t *bytes) {
    if (!bytes || !mlp_dims_ok(d_in, width, d_out, max_batch)) return QP_ERR_ARG;
    *bytes = mlp_layout(nullptr, d_in, width, d_out, max_batch, nullptr);
    return QP_OK;
}

qp_status qp_mlp_create(int d_in, int width, int d_out, int max_batch, void *d_ws, size_t bytes, void *stream,
                        qp_mlp **out) {
    if (!out) return QP_ERR_ARG;
    *out = nullptr;
    if (!mlp_dims_ok(d_in, width, d_out, max_batch) || !d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u))
        return QP_ERR_ARG;
    const size_t need = mlp_layout(nullptr, d_in, width, d_out, max_batch, nullptr);
    if (bytes < need) return QP_ERR_OOM;
    qp_mlp *m = new (std::nothrow) qp_mlp();
    if (!m) return QP_ERR_OOM;
    m->ws = static_cast<char *>(d_ws);
    m->bytes = bytes;
    m->stream = static_cast<cudaStream_t>(stream);
    mlp_layout(m, d_in, width, d_out, max_batch, m->ws);
    // zero everything once: paddings of the BF16 buffers stay zero for good
    if (cudaMemsetAsync(m->ws, 0, need, m->stream) != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess) {
        delete m;
        return QP_ERR_CUDA;
    }
    *out = m;
    return QP_OK;
}

void qp_mlp_destroy(qp_mlp *m) {
    if (!m) return;
    if (m->roll_exec) cudaGraphExecDestroy(m->roll_exec);
    if (m->roll_exec_rem) cudaGraphExecDestroy(m->roll_exec_rem);
    delete m;
}

qp_status qp_mlp_num_params(const qp_mlp *m, int64_t *n) {
    if (!m || !n) return QP_ERR_ARG;
    *n = m->npar;
    return QP_OK;
}

qp_status qp_mlp_set_params(qp_mlp *m, const float *h_params) {
    if (!m || !h_params) return QP_ERR_ARG;
    for (long long i = 0; i < m->npar; ++i)
        if (!std::isfinite(h_params[i])) return mfail(m, QP_ERR_ARG, "parameters must be finite");
    if (cudaMemcpyAsync(m->par, h_params, m->npar * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "copy");
    cudaMemsetAsync(m->mom, 0, m->npar * 4, m->stream);
    cudaMemsetAsync(m->vel, 0, m->npar * 4, m->stream);
    for (int l = 0; l < 3; ++l) k_round_weights<<<64, 256, 0, m->stream>>>(weight_block(m, l, true));
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "set_params");
    m->step = 0;
    return QP_OK;
}

qp_status qp_mlp_get_params(qp_mlp *m, float *h_params) {
    if (!m || !h_params) return QP_ERR_ARG;
    if (cudaMemcpyAsync(h_params, m->par, m->npar * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "get_params");
    return QP_OK;
}

qp_status qp_mlp_forward(qp_mlp *m, const float *d_x, int batch, float *d_y) {
    if (!m || !d_x || !d_y || batch < 1 || batch > m->max_batch) return QP_ERR_ARG;
    if (forward(m, d_x, batch) != cudaSuccess) return mfail(m, QP_ERR_CUDA, "forward");
    if (cudaMemcpyAsync(d_y, m->y, (size_t)batch * m->d_out * 4, cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "copy");
    return QP_OK;
}

qp_status qp_mlp_gradients(qp_mlp *m, const float *d_x, const float *d_t, int batch, float *h_grads, double *loss) {
    if (!m || !d_x || !d_t || batch < 1 || batch > m->max_batch) return QP_ERR_ARG;
    if (clear_transposed(m, batch) != cudaSuccess || forward(m, d_x, batch) != cudaSuccess ||
        backward(m, d_t, batch) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "forward/backward");
    if (h_grads && cudaMemcpyAsync(h_grads, m->grad, m->npar * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "copy");
    if (loss && cudaMemcpyAsync(loss, m->loss, 8, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "copy");
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mfail(m, QP_ERR_CUDA, "sync");
    return QP_OK;
}

qp_status qp_mlp_train_step(qp_mlp *m, const float *d_x, const float *d_t, int batch, float lr, float beta1, float beta2,
                            float eps, double *loss) {
    if (!m || !d_x || !d_t || batch < 1 || batch > m->max_batch) return QP_ERR_ARG;
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return mfail(m, QP_ERR_ARG, "bad Adam hyper-parameters");
    if (clear_transposed(m, batch) != cudaSuccess || forward(m, d_x, batch) != cudaSuccess ||
        backward(m, d_t, batch) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "forward/backward");
    ++m->step;
    const float bc1 = 1.f - powf(beta1, (float)m->step), bc2 = 1.f - powf(beta2, (float)m->step);
    for (int l = 0; l < 3; ++l) {
        k_adam<<<128, 256, 0, m->stream>>>(weight_block(m, l, true), lr, beta1, beta2, eps, bc1, bc2);
        k_adam<<<8, 256, 0, m->stream>>>(bias_block(m, l), lr, beta1, beta2, eps, bc1, bc2);
    }
    if (cudaGetLastError() != cudaSuccess) return mfail(m, QP_ERR_CUDA, "adam");
    if (loss) {
        if (cudaMemcpyAsync(loss, m->loss, 8, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaStreamSynchronize(m->stream) != cudaSuccess)
            return mfail(m, QP_ERR_CUDA, "loss");
    }
    return QP_OK;
}

qp_status qp_surrogate_windows(const double *d_rho, int n_inst, int L, const float *d_par, int n_par, int t_begin,
                               int t_end, int inst0, int ninst_used, float out_scale, float *d_x, float *d_tgt,
                               void *stream) {
    if (!d_rho || !d_par || !d_x || !d_tgt || L < 1 || n_par < 0 || t_begin < L || t_end <= t_begin || inst0 < 0 ||
        ninst_used < 1 || inst0 + ninst_used > n_inst || !(out_scale > 0.f))
        return QP_ERR_ARG;
    k_windows<<<256, 256, 0, static_cast<cudaStream_t>(stream)>>>(reinterpret_cast<const double2 *>(d_rho), n_inst, L,
                                                                  d_par, n_par, t_begin, t_end, inst0, ninst_used,
                                                                  out_scale, d_x, d_tgt);
    return cudaGetLastError() == cudaSuccess ? QP_OK : QP_ERR_CUDA;
}

qp_status qp_surrogate_rollout(qp_mlp *m, float *d_hist, int n, int T, int L, const float *d_par, int n_par,
                               int t_from, int t_to, float out_scale, float *d_xbuf, float *d_ybuf) {
    if (!m || !d_hist || !d_par || !d_xbuf || !d_ybuf || n < 1 || n > m->max_batch || L < 1 || t_from < L ||
        t_to > T || t_to < t_from || 8 * L + n_par != m->d_in || m->d_out != 8 || !(out_scale > 0.f))
        return QP_ERR_ARG;
    (void)d_ybuf;
    const int nsteps = t_to - t_from;
    if (nsteps == 0) return QP_OK;
    // one block for every step when the batch is one or two m16 tiles and
    // the first layer's weights fit shared memory
    const int MT = (n + 15) / 16;
    const size_t kSmemMax = (size_t)227 * 1024;
    const bool ring = roll_smem_bytes(MT, m->width, m->K1, m->Kw, n, L, true) <= kSmemMax;
    const size_t fsm = roll_smem_bytes(MT, m->width, m->K1, m->Kw, n, L, ring);
    const bool fused_ok = MT <= 2 && m->d_out == 8 && m->width % 8 == 0 && fsm <= kSmemMax;
    if (m->roll_mode == QP_ROLLOUT_FUSED && !fused_ok)
        return mfail(m, QP_ERR_ARG, "fused rollout: needs n <= 32, 8 outputs and the first layer in shared memory");
    if (fused_ok && m->roll_mode != QP_ROLLOUT_GRAPH) {
        RollArgs ra;
        ra.hist = d_hist;
        ra.par = d_par;
        ra.w1t = m->WbT[0];
        ra.w2t = m->WbT[1];
        ra.w3t = m->WbT[2];
        ra.b1 = m->b[0];
        ra.b2 = m->b[1];
        ra.b3 = m->b[2];
        ra.n = n;
        ra.T = T;
        ra.L = L;
        ra.n_par = n_par;
        ra.d_in = m->d_in;
        ra.width = m->width;
        ra.K1 = m->K1;
        ra.Kw = m->Kw;
        ra.t_from = t_from;
        ra.t_to = t_to;
        ra.ring = ring ? 1 : 0;
        ra.out_scale = out_scale;
        const void *fn = MT == 1 ? (const void *)k_rollout_fused<1> : (const void *)k_rollout_fused<2>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm) != cudaSuccess)
            return mfail(m, QP_ERR_CUDA, "fused rollout set-up");
        if (MT == 1) k_rollout_fused<1><<<2, kRollThreads, fsm, m->stream>>>(ra);   // one cluster of two
        else k_rollout_fused<2><<<2, kRollThreads, fsm, m->stream>>>(ra);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess)
            return mfail(m, QP_ERR_CUDA, "fused rollout");
        return QP_OK;
    }
    // one rollout step: features packed for the first layer, the network,
    // the update (which advances the device step index)
    auto one_step = [&]() -> cudaError_t {
        k_rollout_pack<<<64, 256, 0, m->stream>>>(d_hist, n, T, L, d_par, n_par, m->tstep, m->xb, m->K1);
        cudaError_t e = forward_layers(m, n);
        if (e != cudaSuccess) return e;
        k_rollout_update<<<(n + 127) / 128, 128, 0, m->stream>>>(d_hist, n, T, m->tstep, m->tdone, m->y, out_scale);
        return cudaGetLastError();
    };
    auto capture = [&](int steps, cudaGraphExec_t *exec) -> cudaError_t {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        for (int k = 0; k < steps && e == cudaSuccess; ++k) e = one_step();
        cudaError_t e2 = cudaStreamEndCapture(m->stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
        if (g) cudaGraphDestroy(g);
        return e;
    };
    // steps are replayed in graphs of up to 32 (the arguments each graph
    // bakes in form its key; a different call captures again)
    const int G = std::min(32, nsteps), rem = nsteps % G;
    const void *key[4] = {d_hist, d_par, d_xbuf, m->ws};
    const int dims[6] = {n, T, L, n_par, G, rem};
    bool same = m->roll_exec && m->roll_scale == out_scale && m->roll_steps == G && m->roll_rem == rem;
    for (int i = 0; i < 4 && same; ++i) same = m->roll_key[i] == key[i];
    for (int i = 0; i < 6 && same; ++i) same = m->roll_dims[i] == dims[i];
    if (cudaMemsetAsync(m->tdone, 0, 4, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(m->tstep, &t_from, 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        return mfail(m, QP_ERR_CUDA, "rollout set-up");
    if (m->stream == nullptr) {   // the legacy default stream cannot be captured: launch step by step
        for (int k = 0; k < nsteps; ++k)
            if (one_step() != cudaSuccess) return mfail(m, QP_ERR_CUDA, "rollout");
        if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mfail(m, QP_ERR_CUDA, "rollout");
        return QP_OK;
    }
    if (!same) {
        if (m->roll_exec) cudaGraphExecDestroy(m->roll_exec);
        if (m->roll_exec_rem) cudaGraphExecDestroy(m->roll_exec_rem);
        m->roll_exec = m->roll_exec_rem = nullptr;
        if (capture(G, &m->roll_exec) != cudaSuccess || (rem && capture(rem, &m->roll_exec_rem) != cudaSuccess))
            return mfail(m, QP_ERR_CUDA, "rollout graph capture");
        m->roll_steps = G;
        m->roll_rem = rem;
        m->roll_scale = out_scale;
        for (int i = 0; i < 4; ++i) m->roll_key[i] = key[i];
        for (int i = 0; i < 6; ++i) m->roll_dims[i] = dims[i];
    }
    for (int k = 0; k < nsteps / G; ++k)
        if (cudaGraphLaunch(m->roll_exec, m->stream) != cudaSuccess) return mfail(m, QP_ERR_CUDA, "rollout graph");
    if (rem && cudaGraphLaunch(m->roll_exec_rem, m->stream) != cudaSuccess) return mfail(m, QP_ERR_CUDA, "rollout graph");
    // the host value t_from is read by the copy before the call returns
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mfail(m, QP_ERR_CUDA, "rollout");
    return cudaGetLastError() == cudaSuccess ? QP_OK : mfail(m, QP_ERR_CUDA, "rollout");
}

qp_status qp_mlp_set_rollout_mode(qp_mlp *m, int mode) {
    if (!m) return QP_ERR_ARG;
    if (mode != QP_ROLLOUT_AUTO && mode != QP_ROLLOUT_GRAPH && mode != QP_ROLLOUT_FUSED)
        return mfail(m, QP_ERR_ARG, "unknown rollout mode");
    m->roll_mode = mode;
    return QP_OK;
}

const char *qp_mlp_last_error(const qp_mlp *m) { return m ? m->err.c_str() : "null model"; }

}  // extern "C"
