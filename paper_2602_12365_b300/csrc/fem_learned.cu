// Learned block preconditioner for the Newton-CG PCG (3D meshes, FP32 CG).
//
// A per-node MLP (36 -> 64 -> 64 -> 6, SiLU hidden layers, BF16 weights and
// activations, FP32 accumulation) corrects block Jacobi.  With D_i the nodal
// diagonal block of the tangent, s_i = tr(D_i)/3, D_i/s_i = C C^T (Cholesky)
// and F = C^-T, the block applied in PCG is
//     M_i = F A A^T F^T / s_i,
// A lower-triangular from the six outputs (softplus(o) + 1e-4 on the
// diagonal), so M_i is SPD for any weights and equals block Jacobi D_i^-1
// when A = I (the initial network).  Prescribed components get identity
// rows and columns.
//
// Inference runs the three layers on the tensor cores with mma.sync
// m16n8k16 (one warp per 16 nodes, the layers chained in registers: the
// accumulator fragments of two adjacent 8-column tiles are the next layer's
// 16-wide A fragment); the epilogue forms M_i per node.  In the Newton
// solve's preconditioner build, features, network and block map run in one
// kernel (lp_precond_kernel), the features staying in shared memory.  The
// network is 3.7 GFLOP per call on 274k nodes; what bounds the kernel is the
// per-node scalar work around it (neighbour sums, logarithms, 128 SiLUs per
// node), so the warp-level MMA is enough.
//
// Training minimises ||H M r - r||^2 / ||r||^2 over states u and residuals
// r of the method's own Newton solves (H = M K(u) M, masked): the forward
// needs one HVP, the backward dL/dz = 2 H (H z - r) / ||r||^2 a second one.
// The weight gradient is a per-node FP32 backward through the block map and
// the MLP (recomputing the forward with the same BF16 roundings as the
// inference), accumulated per block in a fixed order; a last kernel adds the
// block partials in block order and takes an Adam step on FP32 master
// weights, then refreshes the BF16 copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fem_b300.h"
#include "fem_internal.h"
#include "fem_kernels.cuh"

namespace {

constexpr int kIn = FEM_LP_FEATURES;  // 36
constexpr int kInPad = 48;            // K of layer 1, a multiple of 16
constexpr int kH = 64;
constexpr int kOut = 6;
// parameter vector (FP32, W[out][in] row-major), the layout of the C API
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH * kIn;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kOut * kH;
constexpr int kParams = kOffB3 + kOut;
static_assert(kParams == FEM_LP_PARAMS, "parameter count");
// BF16 inference copies: row strides padded by 8 against bank conflicts
constexpr int kS1 = kInPad + 8;  // 56
constexpr int kS2 = kH + 8;      // 72
constexpr int kBf16Elems = kH * kS1 + kH * kS2 + 8 * kS2;
constexpr int kBiasFloats = kH + kH + 8;

constexpr int kInferThreads = 128;
constexpr int kGradThreads = 256;
constexpr int kGradTile = 32;  // nodes per backward tile
constexpr int kGradBlocks = 296;
constexpr int kVecT = 256;
constexpr int kRedBlocks = 296;

fem_status fail(fem_status s, const std::string& msg) { return femi::set_error(s, msg); }

#define CUDA_TRY(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(FEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define FEM_TRY(call)                \
    do {                             \
        fem_status s_ = (call);      \
        if (s_ != FEM_OK) return s_; \
    } while (0)

// ---------------------------------------------------------------------------
// shared device helpers
// ---------------------------------------------------------------------------
// SiLU of the hidden layers with the fast exponential and division
// intrinsics (about 1e-6 relative; each result is rounded to BF16 at once,
// a 4e-3 step): the network is issue-bound on these, 128 per node.  Below
// -87 the denominator overflows and the quotient is zero, as SiLU is there
// to FP32 precision.  Inference and the training's recomputed forward call
// the same function.
__device__ __forceinline__ float silu(float x) { return __fdividef(x, 1.0f + __expf(-x)); }
__device__ __forceinline__ float dsilu(float x) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-x));
    return s * (1.0f + x * (1.0f - s));
}
__device__ __forceinline__ float softplus(float x) { return x > 20.0f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid(float x) { return 1.0f / (1.0f + expf(-x)); }
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (lower column) in the low half
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// F = C^-T with D/s = C C^T (FP32); false if D/s is not SPD
__device__ __forceinline__ bool lp_factor(const float (&Di)[9], float (&Fm)[3][3], float& s) {
    s = (Di[0] + Di[4] + Di[8]) * (1.0f / 3.0f);
    if (!(s > 0.0f)) return false;
    const float is = 1.0f / s;
    float C[3][3] = {}, Ci[3][3] = {};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float t = Di[i * 3 + j] * is;
#pragma unroll
            for (int k = 0; k < j; ++k) t -= C[i][k] * C[j][k];
            if (i == j) {
                if (!(t > 0.0f)) return false;
                C[i][i] = sqrtf(t);
            } else {
                C[i][j] = t / C[j][j];
            }
        }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float t = (i == j) ? 1.0f : 0.0f;
#pragma unroll
            for (int k = 0; k < i; ++k) t -= C[i][k] * Ci[k][j];
            Ci[i][j] = t / C[i][i];
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Fm[i][j] = Ci[j][i];
    return true;
}

__device__ __forceinline__ void lp_A(const float (&o)[6], float (&A)[3][3]) {
    A[0][0] = softplus(o[0]) + 1e-4f;
    A[0][1] = 0.f;
    A[0][2] = 0.f;
    A[1][0] = o[1];
    A[1][1] = softplus(o[2]) + 1e-4f;
    A[1][2] = 0.f;
    A[2][0] = o[3];
    A[2][1] = o[4];
    A[2][2] = softplus(o[5]) + 1e-4f;
}

// M = F A A^T F^T / s with identity rows/columns on prescribed components
__device__ __forceinline__ void lp_block(const float (&Di)[9], uint8_t mask, const float (&o)[6], float* M) {
    float Fm[3][3], A[3][3], s;
    float out[9];
    if (!lp_factor(Di, Fm, s)) {
#pragma unroll
        for (int k = 0; k < 9; ++k) out[k] = (k % 4 == 0) ? 1.f : 0.f;
    } else {
        lp_A(o, A);
        float FA[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) FA[i][j] = Fm[i][0] * A[0][j] + Fm[i][1] * A[1][j] + Fm[i][2] * A[2][j];
        const float is = 1.0f / s;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                out[i * 3 + j] = (FA[i][0] * FA[j][0] + FA[i][1] * FA[j][1] + FA[i][2] * FA[j][2]) * is;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if ((mask >> c) & 1)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    out[c * 3 + k] = (k == c) ? 1.f : 0.f;
                    out[k * 3 + c] = (k == c) ? 1.f : 0.f;
                }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) M[k] = out[k];
}

// ---------------------------------------------------------------------------
// features: 36 per node (BF16, padded to 48)
//   [0,9)   D_i / s_i
//   [9,18)  mean over neighbour nodes of D_j, / s_i
//   [18,27) mean absolute deviation of the neighbours' D_j, / s_i
//           (these 27 compressed as sign(x) ln(1 + |x|))
//   27 ln mean mu, 28 ln(mean lambda / mean mu), 29 valence / 24
//   [30,33) Dirichlet bits, [33,36) ln(D_i,cc / s_i)
// ---------------------------------------------------------------------------
// the 36 features of node n as 18 BF16 pairs (all zero when D_n has no
// positive trace), and D_n itself.  The neighbours' blocks are loaded
// kNb at a time (their loads in flight together) and added in list order.
constexpr int kNb = 4;
__device__ __forceinline__ void lp_node_features(int64_t n, const float* D, const float* D8, const int64_t* ptr,
                                                 const int32_t* idx, const float* stats, const uint8_t* node_mask,
                                                 uint32_t (&xw)[kIn / 2], float (&Di)[9]) {
    float f[kIn];
#pragma unroll
    for (int k = 0; k < 9; ++k) Di[k] = D[n * 9 + k];
    const float s = (Di[0] + Di[4] + Di[8]) * (1.0f / 3.0f);
    const bool ok = s > 0.0f && isfinite(s);
    const float is = ok ? 1.0f / s : 0.0f;
    float mean[9] = {}, dev[9] = {};
    const int64_t j0 = ptr[n], j1 = ptr[n + 1];
    // one pass over the neighbour list: kNb blocks in flight, then their adds
    // (dv = 1: sum of D_j; dv = 2: sum of |D_j - mean|)
    auto pass = [&](int dv) {
        for (int64_t j = j0; j < j1; j += kNb) {
            int32_t q[kNb];
#pragma unroll
            for (int b = 0; b < kNb; ++b) q[b] = j + b < j1 ? idx[j + b] : -1;
            // the nodal blocks are symmetric (the block diagonal is written
            // from its six distinct entries): D8 holds those, 16-byte aligned
            float t[kNb][9];
#pragma unroll
            for (int b = 0; b < kNb; ++b) {
                float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
                if (q[b] >= 0) {
                    lo = reinterpret_cast<const float4*>(D8)[2 * (int64_t)q[b]];
                    hi = reinterpret_cast<const float4*>(D8)[2 * (int64_t)q[b] + 1];
                }
                t[b][0] = lo.x, t[b][1] = lo.y, t[b][2] = lo.z;
                t[b][3] = lo.y, t[b][4] = lo.w, t[b][5] = hi.x;
                t[b][6] = lo.z, t[b][7] = hi.x, t[b][8] = hi.y;
            }
#pragma unroll
            for (int b = 0; b < kNb; ++b) {
                if (q[b] < 0) break;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    if (dv == 1)
                        mean[k] += t[b][k];
                    else
                        dev[k] += fabsf(t[b][k] - mean[k]);
                }
            }
        }
    };
    pass(1);
    const float inb = j1 > j0 ? 1.0f / (float)(j1 - j0) : 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) mean[k] *= inb;
    pass(2);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        f[k] = Di[k] * is;
        f[9 + k] = mean[k] * is;
        f[18 + k] = dev[k] * inb * is;
    }
    // block ratios span orders of magnitude at boundary and
    // high-contrast nodes: compress them as sign(x) ln(1 + |x|), by the
    // branch-free FP32 logarithm (exponent split and artanh series, a few
    // ulps for every finite |x|; the feature is then rounded to BF16)
#pragma unroll
    for (int k = 0; k < 27; ++k) f[k] = copysignf(fem::vlog1p_bf(fabsf(f[k])), f[k]);
    f[27] = stats[n * 3 + 0];
    f[28] = stats[n * 3 + 1];
    f[29] = stats[n * 3 + 2];
    const uint8_t m = node_mask[n];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        f[30 + c] = ((m >> c) & 1) ? 1.0f : 0.0f;
        f[33 + c] = ok ? logf(Di[c * 4] * is) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kIn; k += 2) xw[k / 2] = ok ? pack_bf16(f[k], f[k + 1]) : 0u;
}

// D8 of every node from its block in D
__global__ void __launch_bounds__(kVecT) lp_pack_kernel(int64_t nn, const float* D, float* D8) {
    for (int64_t n = blockIdx.x * (int64_t)kVecT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVecT) {
        const float* b = D + n * 9;
        reinterpret_cast<float4*>(D8)[2 * n] = make_float4(b[0], b[1], b[2], b[4]);
        reinterpret_cast<float4*>(D8)[2 * n + 1] = make_float4(b[5], b[8], 0.f, 0.f);
    }
}

__global__ void __launch_bounds__(kVecT) lp_features_kernel(int64_t nn, const float* D, const float* D8,
                                                            const int64_t* ptr,
                                                            const int32_t* idx, const float* stats,
                                                            const uint8_t* node_mask, __nv_bfloat16* X) {
    for (int64_t n = blockIdx.x * (int64_t)kVecT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVecT) {
        uint32_t xw[kIn / 2];
        float Di[9];
        lp_node_features(n, D, D8, ptr, idx, stats, node_mask, xw, Di);
        uint32_t* dst = reinterpret_cast<uint32_t*>(X + n * kInPad);
#pragma unroll
        for (int k = 0; k < kIn / 2; ++k) dst[k] = xw[k];
#pragma unroll
        for (int k = kIn / 2; k < kInPad / 2; ++k) dst[k] = 0u;
    }
}

// ---------------------------------------------------------------------------
// inference: BF16 tensor-core MLP, then the block map
// ---------------------------------------------------------------------------
struct InferW {
    const __nv_bfloat16* w;  // [w1 64 x kS1 | w2 64 x kS2 | w3 8 x kS2]
    const float* b;          // [b1 64 | b2 64 | b3 8]
};

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// The network on one tile of 16 nodes (one warp, mma.sync m16n8k16): a1 holds
// the tile's layer-1 A fragments (k blocks of 16 over the 48 padded inputs),
// the weights and biases are in shared memory; o3 gets the lane's outputs
// (rows g and g + 8, columns 2t and 2t + 1; columns 6 and 7 are zero rows).
// The accumulator fragments of two adjacent 8-column tiles are the next
// layer's 16-wide A fragment, so the layers chain in registers.
__device__ __forceinline__ void lp_mlp16(const uint32_t (&a1)[kInPad / 16][4], const __nv_bfloat16* sW1,
                                         const __nv_bfloat16* sW2, const __nv_bfloat16* sW3, const float* sb1,
                                         const float* sb2, const float* sb3, int g, int t, float (&o3)[4]) {
    // layer 1: [16 x 48] x [48 x 64]
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        acc[j][0] = acc[j][2] = sb1[8 * j + 2 * t];
        acc[j][1] = acc[j][3] = sb1[8 * j + 2 * t + 1];
    }
#pragma unroll
    for (int kk = 0; kk < kInPad / 16; ++kk)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const __nv_bfloat16* wr = sW1 + (8 * j + g) * kS1 + 16 * kk + 2 * t;
            mma_bf16(acc[j], a1[kk], ld32(wr), ld32(wr + 8));
        }
    // SiLU, BF16: the accumulators of n-tiles 2kk, 2kk+1 are layer 2's A fragment kk
    uint32_t ah[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        ah[kk][0] = pack_bf16(silu(acc[2 * kk][0]), silu(acc[2 * kk][1]));
        ah[kk][1] = pack_bf16(silu(acc[2 * kk][2]), silu(acc[2 * kk][3]));
        ah[kk][2] = pack_bf16(silu(acc[2 * kk + 1][0]), silu(acc[2 * kk + 1][1]));
        ah[kk][3] = pack_bf16(silu(acc[2 * kk + 1][2]), silu(acc[2 * kk + 1][3]));
    }
    // layer 2: [16 x 64] x [64 x 64]
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        acc[j][0] = acc[j][2] = sb2[8 * j + 2 * t];
        acc[j][1] = acc[j][3] = sb2[8 * j + 2 * t + 1];
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const __nv_bfloat16* wr = sW2 + (8 * j + g) * kS2 + 16 * kk + 2 * t;
            mma_bf16(acc[j], ah[kk], ld32(wr), ld32(wr + 8));
        }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        ah[kk][0] = pack_bf16(silu(acc[2 * kk][0]), silu(acc[2 * kk][1]));
        ah[kk][1] = pack_bf16(silu(acc[2 * kk][2]), silu(acc[2 * kk][3]));
        ah[kk][2] = pack_bf16(silu(acc[2 * kk + 1][0]), silu(acc[2 * kk + 1][1]));
        ah[kk][3] = pack_bf16(silu(acc[2 * kk + 1][2]), silu(acc[2 * kk + 1][3]));
    }
    // layer 3: [16 x 64] x [64 x 8] (outputs 6, 7 are zero rows)
    o3[0] = sb3[2 * t], o3[1] = sb3[2 * t + 1], o3[2] = sb3[2 * t], o3[3] = sb3[2 * t + 1];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const __nv_bfloat16* wr = sW3 + g * kS2 + 16 * kk + 2 * t;
        mma_bf16(o3, ah[kk], ld32(wr), ld32(wr + 8));
    }
}

__global__ void __launch_bounds__(kInferThreads) lp_infer_kernel(int64_t nn, const __nv_bfloat16* X, const float* D,
                                                                 const uint8_t* node_mask, InferW W, float* Minv) {
    __shared__ __align__(16) __nv_bfloat16 sW[kBf16Elems];
    __shared__ float sB[kBiasFloats];
    __shared__ float sOut[kInferThreads / 32][16][8];
    for (int i = threadIdx.x; i < kBf16Elems; i += kInferThreads) sW[i] = W.w[i];
    for (int i = threadIdx.x; i < kBiasFloats; i += kInferThreads) sB[i] = W.b[i];
    __syncthreads();
    const __nv_bfloat16* sW1 = sW;
    const __nv_bfloat16* sW2 = sW + kH * kS1;
    const __nv_bfloat16* sW3 = sW2 + kH * kS2;
    const float* sb1 = sB;
    const float* sb2 = sB + kH;
    const float* sb3 = sB + 2 * kH;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t n_tiles = (nn + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * (kInferThreads / 32) + warp; tile < n_tiles;
         tile += (int64_t)gridDim.x * (kInferThreads / 32)) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        // layer 1's A fragments of the tile from the features in global memory
        uint32_t a1[kInPad / 16][4];
#pragma unroll
        for (int kk = 0; kk < kInPad / 16; ++kk) {
            a1[kk][0] = r0 < nn ? ld32(X + r0 * kInPad + 16 * kk + 2 * t) : 0u;
            a1[kk][1] = r1 < nn ? ld32(X + r1 * kInPad + 16 * kk + 2 * t) : 0u;
            a1[kk][2] = r0 < nn ? ld32(X + r0 * kInPad + 16 * kk + 8 + 2 * t) : 0u;
            a1[kk][3] = r1 < nn ? ld32(X + r1 * kInPad + 16 * kk + 8 + 2 * t) : 0u;
        }
        float o3[4];
        lp_mlp16(a1, sW1, sW2, sW3, sb1, sb2, sb3, g, t, o3);
        sOut[warp][g][2 * t] = o3[0];
        sOut[warp][g][2 * t + 1] = o3[1];
        sOut[warp][g + 8][2 * t] = o3[2];
        sOut[warp][g + 8][2 * t + 1] = o3[3];
        __syncwarp();
        const int64_t n = tile * 16 + lane;
        if (lane < 16 && n < nn) {
            float o[6], Di[9];
#pragma unroll
            for (int k = 0; k < 6; ++k) o[k] = sOut[warp][lane][k];
#pragma unroll
            for (int k = 0; k < 9; ++k) Di[k] = D[n * 9 + k];
            lp_block(Di, node_mask[n], o, Minv + n * 9);
        }
        __syncwarp();
    }
}

// Features, network and block map in one pass (the preconditioner build of
// a Newton iteration): each warp takes 32 nodes at a time, one per lane; the
// lane's features go to its row of the warp's tile in shared memory (BF16,
// zero-padded to 48 inputs), the network runs on the tile's two 16-node
// halves, and each lane applies the block map to its own node with the D_n
// it loaded for the features.  The features never go through global memory;
// the arithmetic is that of lp_features_kernel followed by lp_infer_kernel.
constexpr int kPrecondThreads = 128;
__global__ void __launch_bounds__(kPrecondThreads, 5) lp_precond_kernel(int64_t nn, const float* D, const float* D8,
                                                                     const int64_t* ptr,
                                                                     const int32_t* idx, const float* stats,
                                                                     const uint8_t* node_mask, InferW W,
                                                                     float* Minv) {
    constexpr int kWarps_ = kPrecondThreads / 32;
    constexpr int kRowWords = kS1 / 2;  // 28 words per row: conflict-free fragment loads
    __shared__ __align__(16) __nv_bfloat16 sW[kBf16Elems];
    __shared__ float sB[kBiasFloats];
    __shared__ __align__(16) uint32_t sX[kWarps_][32][kRowWords];
    __shared__ float sOut[kWarps_][32][8];
    for (int i = threadIdx.x; i < kBf16Elems; i += kPrecondThreads) sW[i] = W.w[i];
    for (int i = threadIdx.x; i < kBiasFloats; i += kPrecondThreads) sB[i] = W.b[i];
    __syncthreads();
    const __nv_bfloat16* sW1 = sW;
    const __nv_bfloat16* sW2 = sW + kH * kS1;
    const __nv_bfloat16* sW3 = sW2 + kH * kS2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t n_groups = (nn + 31) / 32;
    for (int64_t grp = (int64_t)blockIdx.x * kWarps_ + warp; grp < n_groups; grp += (int64_t)gridDim.x * kWarps_) {
        const int64_t n = grp * 32 + lane;
        uint32_t* row = sX[warp][lane];
        float Di[9] = {};
        if (n < nn) {
            uint32_t xw[kIn / 2];
            lp_node_features(n, D, D8, ptr, idx, stats, node_mask, xw, Di);
#pragma unroll
            for (int k = 0; k < kIn / 2; ++k) row[k] = xw[k];
        } else {
#pragma unroll
            for (int k = 0; k < kIn / 2; ++k) row[k] = 0u;
        }
#pragma unroll
        for (int k = kIn / 2; k < kInPad / 2; ++k) row[k] = 0u;
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // rows 16h .. 16h + 15 of the tile
            uint32_t a1[kInPad / 16][4];
#pragma unroll
            for (int kk = 0; kk < kInPad / 16; ++kk) {
                a1[kk][0] = sX[warp][16 * h + g][8 * kk + t];
                a1[kk][1] = sX[warp][16 * h + g + 8][8 * kk + t];
                a1[kk][2] = sX[warp][16 * h + g][8 * kk + 4 + t];
                a1[kk][3] = sX[warp][16 * h + g + 8][8 * kk + 4 + t];
            }
            float o3[4];
            lp_mlp16(a1, sW1, sW2, sW3, sB, sB + kH, sB + 2 * kH, g, t, o3);
            sOut[warp][16 * h + g][2 * t] = o3[0];
            sOut[warp][16 * h + g][2 * t + 1] = o3[1];
            sOut[warp][16 * h + g + 8][2 * t] = o3[2];
            sOut[warp][16 * h + g + 8][2 * t + 1] = o3[3];
        }
        __syncwarp();
        if (n < nn) {
            float o[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) o[k] = sOut[warp][lane][k];
            lp_block(Di, node_mask[n], o, Minv + n * 9);
        }
        __syncwarp();  // the tile's rows and outputs are rewritten by the next group
    }
}

// ---------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------
// z_i = M_i r_i
__global__ void lp_apply_kernel(int64_t nn, const float* Minv, const float* r, float* z) {
    for (int64_t n = blockIdx.x * (int64_t)kVecT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVecT) {
        const float* M = Minv + n * 9;
        const float x = r[n * 3], y = r[n * 3 + 1], w = r[n * 3 + 2];
#pragma unroll
        for (int i = 0; i < 3; ++i) z[n * 3 + i] = M[i * 3] * x + M[i * 3 + 1] * y + M[i * 3 + 2] * w;
    }
}

// e = q - r (q = H z); block partials of r.r, e.e, z.q, r.z in FP64
__global__ void lp_residual_kernel(int64_t n, const float* q, const float* r, const float* z, float* e,
                                   double* partial) {
    __shared__ double sh[kVecT / 32][4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)kVecT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecT) {
        const float d = q[i] - r[i];
        e[i] = d;
        v[0] = fma((double)r[i], (double)r[i], v[0]);
        v[1] = fma((double)d, (double)d, v[1]);
        v[2] = fma((double)z[i], (double)q[i], v[2]);
        v[3] = fma((double)r[i], (double)z[i], v[3]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[threadIdx.x >> 5][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kVecT / 32; ++w)
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] += sh[w][k];
#pragma unroll
        for (int k = 0; k < 4; ++k) partial[blockIdx.x * 4 + k] = v[k];
    }
}

// one block: sum the partials in block order.  loss3 = (r.r, unused, loss):
// residual loss e.e / r.r; energy loss 1 + (z.Hz - 2 r.z) / r.r, i.e.
// ||H z - r||^2 in the H^-1 norm, shifted by r^T H^-1 r / r.r
__global__ void lp_loss_kernel(int nb, const double* partial, int kind, double* loss3) {
    if (threadIdx.x == 0) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < 4; ++k) v[k] += partial[b * 4 + k];
        loss3[0] = v[0];
        loss3[1] = 0.0;
        if (!(v[0] > 0.0))
            loss3[2] = 0.0;
        else
            loss3[2] = kind == FEM_LP_LOSS_ENERGY ? 1.0 + (v[2] - 2.0 * v[3]) / v[0] : v[1] / v[0];
    }
}

// g *= 2 / r.r
__global__ void lp_scale_kernel(int64_t n, float* g, const double* loss3) {
    const float c = loss3[0] > 0.0 ? (float)(2.0 / loss3[0]) : 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)kVecT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecT) g[i] *= c;
}

struct GradSmem {
    float W1[kH][kIn + 1], b1[kH], W2[kH][kH + 1], b2[kH], W3[kOut][kH + 1], b3[8];
    float X[kGradTile][kIn];
    float Z1[kGradTile][kH], H1[kGradTile][kH], Z2[kGradTile][kH], H2[kGradTile][kH];
    float dZ1[kGradTile][kH], dZ2[kGradTile][kH];
    float O[kGradTile][8], dO[kGradTile][8];
};

// Per-node backward of L = sum_i g_i . (M_i r_i) through the block map and
// the MLP; each block accumulates its nodes' weight gradients in a fixed
// order and stores them to partial[blockIdx.x][kParams].
__global__ void __launch_bounds__(kGradThreads) lp_grad_kernel(int64_t nn, const __nv_bfloat16* X, const float* D,
                                                               const uint8_t* node_mask, const float* r,
                                                               const float* gz, InferW W, float* partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
    const int tid = threadIdx.x;
    // the weights exactly as the inference sees them (BF16 values, FP32 biases)
    for (int i = tid; i < kH * kIn; i += kGradThreads)
        S.W1[i / kIn][i % kIn] = __bfloat162float(W.w[(i / kIn) * kS1 + i % kIn]);
    for (int i = tid; i < kH * kH; i += kGradThreads)
        S.W2[i / kH][i % kH] = __bfloat162float(W.w[kH * kS1 + (i / kH) * kS2 + i % kH]);
    for (int i = tid; i < kOut * kH; i += kGradThreads)
        S.W3[i / kH][i % kH] = __bfloat162float(W.w[kH * kS1 + kH * kS2 + (i / kH) * kS2 + i % kH]);
    for (int i = tid; i < kH; i += kGradThreads) {
        S.b1[i] = W.b[i];
        S.b2[i] = W.b[kH + i];
    }
    if (tid < 8) S.b3[tid] = W.b[2 * kH + tid];
    // per-thread gradient accumulators: dW2 (16), dW1 (9), dW3 (2), one bias
    float aW2[16] = {}, aW1[9] = {}, aW3[2] = {}, aB = 0.f;
    __syncthreads();
    const int64_t n_tiles = (nn + kGradTile - 1) / kGradTile;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t base = tile * kGradTile;
        for (int i = tid; i < kGradTile * kIn; i += kGradThreads) {
            const int n = i / kIn, k = i % kIn;
            S.X[n][k] = base + n < nn ? __bfloat162float(X[(base + n) * kInPad + k]) : 0.f;
        }
        __syncthreads();
        // forward (the same roundings as the tensor-core inference)
        {
            const int j = tid % kH;
            for (int n = tid / kH; n < kGradTile; n += kGradThreads / kH) {
                float z = S.b1[j];
                for (int k = 0; k < kIn; ++k) z = fmaf(S.W1[j][k], S.X[n][k], z);
                S.Z1[n][j] = z;
                S.H1[n][j] = bf16r(silu(z));
            }
        }
        __syncthreads();
        {
            const int j = tid % kH;
            for (int n = tid / kH; n < kGradTile; n += kGradThreads / kH) {
                float z = S.b2[j];
                for (int k = 0; k < kH; ++k) z = fmaf(S.W2[j][k], S.H1[n][k], z);
                S.Z2[n][j] = z;
                S.H2[n][j] = bf16r(silu(z));
            }
        }
        __syncthreads();
        if (tid < kGradTile * kOut) {
            const int n = tid / kOut, o = tid % kOut;
            float z = S.b3[o];
            for (int k = 0; k < kH; ++k) z = fmaf(S.W3[o][k], S.H2[n][k], z);
            S.O[n][o] = z;
        }
        __syncthreads();
        // block map backward: G = g r^T (masked), dL/dB = F^T G F / s,
        // dL/dA = (H + H^T) A, through softplus on the diagonal
        if (tid < kGradTile) {
            const int64_t n = base + tid;
            float dO[6] = {0, 0, 0, 0, 0, 0};
            if (n < nn) {
                float Di[9], Fm[3][3], s;
#pragma unroll
                for (int k = 0; k < 9; ++k) Di[k] = D[n * 9 + k];
                if (lp_factor(Di, Fm, s)) {
                    float o[6], A[3][3];
#pragma unroll
                    for (int k = 0; k < 6; ++k) o[k] = S.O[tid][k];
                    lp_A(o, A);
                    const uint8_t m = node_mask[n];
                    float G[3][3];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const bool fixed = ((m >> i) & 1) || ((m >> j) & 1);
                            G[i][j] = fixed ? 0.f : gz[n * 3 + i] * r[n * 3 + j];
                        }
                    float FtG[3][3], Hm[3][3], Wm[3][3];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j) FtG[i][j] = Fm[0][i] * G[0][j] + Fm[1][i] * G[1][j] + Fm[2][i] * G[2][j];
                    const float is = 1.0f / s;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            Hm[i][j] = (FtG[i][0] * Fm[0][j] + FtG[i][1] * Fm[1][j] + FtG[i][2] * Fm[2][j]) * is;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            Wm[i][j] = (Hm[i][0] + Hm[0][i]) * A[0][j] + (Hm[i][1] + Hm[1][i]) * A[1][j] +
                                       (Hm[i][2] + Hm[2][i]) * A[2][j];
                    dO[0] = Wm[0][0] * sigmoid(o[0]);
                    dO[1] = Wm[1][0];
                    dO[2] = Wm[1][1] * sigmoid(o[2]);
                    dO[3] = Wm[2][0];
                    dO[4] = Wm[2][1];
                    dO[5] = Wm[2][2] * sigmoid(o[5]);
                }
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) S.dO[tid][k] = dO[k];
        }
        __syncthreads();
        // MLP backward (straight through the BF16 roundings)
        {
            const int j = tid % kH;
            for (int n = tid / kH; n < kGradTile; n += kGradThreads / kH) {
                float d = 0.f;
#pragma unroll
                for (int o = 0; o < kOut; ++o) d = fmaf(S.W3[o][j], S.dO[n][o], d);
                S.dZ2[n][j] = d * dsilu(S.Z2[n][j]);
            }
        }
        __syncthreads();
        {
            const int j = tid % kH;
            for (int n = tid / kH; n < kGradTile; n += kGradThreads / kH) {
                float d = 0.f;
                for (int i = 0; i < kH; ++i) d = fmaf(S.W2[i][j], S.dZ2[n][i], d);
                S.dZ1[n][j] = d * dsilu(S.Z1[n][j]);
            }
        }
        __syncthreads();
        // weight gradients of this tile, nodes in order
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = tid + kGradThreads * q, i = e / kH, j = e % kH;
            float a = aW2[q];
            for (int n = 0; n < kGradTile; ++n) a = fmaf(S.dZ2[n][i], S.H1[n][j], a);
            aW2[q] = a;
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int e = tid + kGradThreads * q, j = e / kIn, k = e % kIn;
            float a = aW1[q];
            for (int n = 0; n < kGradTile; ++n) a = fmaf(S.dZ1[n][j], S.X[n][k], a);
            aW1[q] = a;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = tid + kGradThreads * q;
            if (e < kOut * kH) {
                const int o = e / kH, k = e % kH;
                float a = aW3[q];
                for (int n = 0; n < kGradTile; ++n) a = fmaf(S.dO[n][o], S.H2[n][k], a);
                aW3[q] = a;
            }
        }
        if (tid < kH) {
            for (int n = 0; n < kGradTile; ++n) aB += S.dZ1[n][tid];
        } else if (tid < 2 * kH) {
            for (int n = 0; n < kGradTile; ++n) aB += S.dZ2[n][tid - kH];
        } else if (tid < 2 * kH + kOut) {
            for (int n = 0; n < kGradTile; ++n) aB += S.dO[n][tid - 2 * kH];
        }
        __syncthreads();
    }
    float* P = partial + (int64_t)blockIdx.x * kParams;
#pragma unroll
    for (int q = 0; q < 16; ++q) P[kOffW2 + tid + kGradThreads * q] = aW2[q];
#pragma unroll
    for (int q = 0; q < 9; ++q) P[kOffW1 + tid + kGradThreads * q] = aW1[q];
#pragma unroll
    for (int q = 0; q < 2; ++q)
        if (tid + kGradThreads * q < kOut * kH) P[kOffW3 + tid + kGradThreads * q] = aW3[q];
    if (tid < kH)
        P[kOffB1 + tid] = aB;
    else if (tid < 2 * kH)
        P[kOffB2 + tid - kH] = aB;
    else if (tid < 2 * kH + kOut)
        P[kOffB3 + tid - 2 * kH] = aB;
}

// BF16 inference copy of the FP32 master parameters
__device__ __forceinline__ void store_infer(int p, float w, __nv_bfloat16* wb, float* bb) {
    if (p < kOffB1) {
        wb[(p / kIn) * kS1 + p % kIn] = __float2bfloat16_rn(w);
    } else if (p < kOffW2) {
        bb[p - kOffB1] = w;
    } else if (p < kOffB2) {
        const int q = p - kOffW2;
        wb[kH * kS1 + (q / kH) * kS2 + q % kH] = __float2bfloat16_rn(w);
    } else if (p < kOffW3) {
        bb[kH + p - kOffB2] = w;
    } else if (p < kOffB3) {
        const int q = p - kOffW3;
        wb[kH * kS1 + kH * kS2 + (q / kH) * kS2 + q % kH] = __float2bfloat16_rn(w);
    } else {
        bb[2 * kH + p - kOffB3] = w;
    }
}

// gradient = sum of the block partials in block order
__global__ void lp_sum_kernel(int nb, const float* partial, float* grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    float g = 0.f;
    for (int b = 0; b < nb; ++b) g += partial[(int64_t)b * kParams + p];
    grad[p] = g;
}

// one block: the gradient's 2-norm (fixed order) and the clipping factor
// min(1, clip / ||g||)
__global__ void lp_clip_kernel(const float* grad, float clip, float* scale) {
    __shared__ double sh[kVecT / 32];
    double a = 0.0;
    for (int p = threadIdx.x; p < kParams; p += kVecT) a = fma((double)grad[p], (double)grad[p], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kVecT / 32; ++w) a += sh[w];
        const double nrm = sqrt(a);
        *scale = (clip > 0.0f && nrm > (double)clip) ? (float)((double)clip / nrm) : 1.0f;
    }
}

// Adam on the FP32 master weights (gradient scaled by the clipping factor),
// then their BF16 inference copy
__global__ void lp_adam_kernel(const float* grad, const float* scale, float* w, float* m, float* v, float lr,
                               float b1, float b2, float eps, float c1, float c2, __nv_bfloat16* wb, float* bb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float g = grad[p] * *scale;
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float wn = w[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    w[p] = wn;
    store_infer(p, wn, wb, bb);
}

__global__ void lp_refresh_kernel(const float* w, __nv_bfloat16* wb, float* bb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kParams) store_infer(p, w[p], wb, bb);
}

int grid_for(int64_t work, int cap) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + kVecT - 1) / kVecT, cap));
}

}  // namespace

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct fem_lp {
    float* w = nullptr;  // FP32 master [kParams]
    float* m = nullptr;  // Adam moments
    float* v = nullptr;
    __nv_bfloat16* wb = nullptr;  // inference copy
    float* bb = nullptr;
    int64_t step = 0;
    int device = 0;
    int loss = FEM_LP_LOSS_RESIDUAL;
    float clip = 1.0f;  // gradient-norm clipping threshold (0: none)
};

namespace femi {
struct LpMeshData {
    int64_t nn = 0;
    int64_t* ptr = nullptr;
    int32_t* idx = nullptr;
    float* stats = nullptr;
    float* D = nullptr;
    // the blocks' distinct entries D00 D01 D02 D11 D12 D22 and two zeros per
    // node: two 16-byte loads per neighbour in the features
    float* D8 = nullptr;
    __nv_bfloat16* X = nullptr;
    float *Minv = nullptr, *z = nullptr, *q = nullptr, *e = nullptr;
    float* partial = nullptr;  // [kGradBlocks * kParams]
    float* grad = nullptr;     // [kParams], then the clipping factor
    double* red = nullptr;     // [kRedBlocks * 4 + 3]
    std::vector<void*> allocs;
};

void lp_mesh_free(fem_mesh* m) {
    if (!m || !m->lp) return;
    for (void* p : m->lp->allocs) cudaFree(p);
    delete m->lp;
    m->lp = nullptr;
}
}  // namespace femi

namespace {

template <typename T>
fem_status dalloc(femi::LpMeshData* d, T** p, size_t n) {
    void* q = nullptr;
    CUDA_TRY(cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)));
    d->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return FEM_OK;
}

// node graph (distinct nodes sharing an element), statistics and workspace
fem_status ensure_mesh(fem_mesh* m, cudaStream_t st) {
    if (m->lp) return FEM_OK;
    if (m->dim != 3) return fail(FEM_ERR_ARG, "the learned preconditioner supports 3D meshes only");
    if (m->precision != FEM_PREC_MIXED) return fail(FEM_ERR_ARG, "the learned preconditioner needs a FEM_PREC_MIXED mesh");
    const int64_t nn = m->info.n_nodes, ne = m->info.n_elems;
    const int nen = m->n_en;
    std::vector<int64_t> cnt((size_t)nn + 1, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < nen; ++a) cnt[m->conn_host[e * nen + a] + 1] += nen - 1;
    for (int64_t i = 0; i < nn; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> all((size_t)std::max<int64_t>(cnt[nn], 1));
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < nen; ++a)
            for (int b = 0; b < nen; ++b)
                if (a != b) all[fill[m->conn_host[e * nen + a]]++] = m->conn_host[e * nen + b];
    std::vector<int64_t> ptr((size_t)nn + 1, 0);
    std::vector<int32_t> idx;
    idx.reserve((size_t)cnt[nn] / 2 + 1);
    for (int64_t i = 0; i < nn; ++i) {
        std::sort(all.begin() + cnt[i], all.begin() + cnt[i + 1]);
        for (int64_t j = cnt[i]; j < cnt[i + 1]; ++j)
            if (j == cnt[i] || all[j] != all[j - 1]) idx.push_back(all[j]);
        ptr[i + 1] = (int64_t)idx.size();
    }
    auto* d = new femi::LpMeshData();
    m->lp = d;
    d->nn = nn;
    FEM_TRY(dalloc(d, &d->ptr, ptr.size()));
    FEM_TRY(dalloc(d, &d->idx, idx.size()));
    FEM_TRY(dalloc(d, &d->stats, m->node_stats.size()));
    CUDA_TRY(cudaMemcpyAsync(d->ptr, ptr.data(), ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d->idx, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d->stats, m->node_stats.data(), m->node_stats.size() * sizeof(float),
                             cudaMemcpyHostToDevice, st));
    FEM_TRY(dalloc(d, &d->D, (size_t)nn * 9));
    FEM_TRY(dalloc(d, &d->D8, (size_t)nn * 8));
    FEM_TRY(dalloc(d, &d->X, (size_t)nn * kInPad));
    FEM_TRY(dalloc(d, &d->Minv, (size_t)nn * 9));
    FEM_TRY(dalloc(d, &d->z, (size_t)nn * 3));
    FEM_TRY(dalloc(d, &d->q, (size_t)nn * 3));
    FEM_TRY(dalloc(d, &d->e, (size_t)nn * 3));
    FEM_TRY(dalloc(d, &d->partial, (size_t)kGradBlocks * kParams));
    FEM_TRY(dalloc(d, &d->grad, (size_t)kParams + 1));
    FEM_TRY(dalloc(d, &d->red, (size_t)kRedBlocks * 4 + 3));
    CUDA_TRY(cudaStreamSynchronize(st));  // host vectors go out of scope
    return FEM_OK;
}

// block diagonal at u (FP32) and the features
fem_status features(fem_mesh* m, const float* u, cudaStream_t st) {
    FEM_TRY(ensure_mesh(m, st));
    femi::LpMeshData* d = m->lp;
    FEM_TRY(femi::run_op(m, FEM_F32, fem::OP_BLOCKDIAG, u, nullptr, d->D, nullptr, 0, st, nullptr));
    lp_pack_kernel<<<grid_for(d->nn, 1184), kVecT, 0, st>>>(d->nn, d->D, d->D8);
    lp_features_kernel<<<grid_for(d->nn, 1184), kVecT, 0, st>>>(d->nn, d->D, d->D8, d->ptr, d->idx, d->stats,
                                                                  m->node_mask, d->X);
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

fem_status infer(const fem_lp* lp, fem_mesh* m, float* Minv, cudaStream_t st) {
    femi::LpMeshData* d = m->lp;
    const int64_t tiles = (d->nn + 15) / 16;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 3) / 4, 148 * 8));
    lp_infer_kernel<<<grid, kInferThreads, 0, st>>>(d->nn, d->X, d->D, m->node_mask, InferW{lp->wb, lp->bb}, Minv);
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

fem_status check_lp(const fem_lp* lp) {
    if (!lp) return fail(FEM_ERR_ARG, "null learned-preconditioner handle");
    return FEM_OK;
}

// deterministic initial weights: W1, W2 ~ N(0, 1/fan_in) from a SplitMix64
// stream (Box-Muller), b1 = b2 = 0, W3 = 0 and b3 with softplus(b3) + 1e-4 = 1
// on the diagonal entries: the initial network is block Jacobi
uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
void initial_params(uint64_t seed, std::vector<float>& w) {
    w.assign(kParams, 0.0f);
    uint64_t s = seed;
    auto normal = [&]() {
        const double u1 = ((splitmix64(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
        const double u2 = (splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int i = 0; i < kH * kIn; ++i) w[kOffW1 + i] = (float)(normal() / std::sqrt((double)kIn));
    for (int i = 0; i < kH * kH; ++i) w[kOffW2 + i] = (float)(normal() / std::sqrt((double)kH));
    const float c = (float)std::log(std::expm1(1.0 - 1e-4));
    w[kOffB3 + 0] = c;
    w[kOffB3 + 2] = c;
    w[kOffB3 + 5] = c;
}

fem_status upload_params(fem_lp* lp, const float* host, cudaStream_t st) {
    CUDA_TRY(cudaMemcpyAsync(lp->w, host, kParams * sizeof(float), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(lp->m, 0, kParams * sizeof(float), st));
    CUDA_TRY(cudaMemsetAsync(lp->v, 0, kParams * sizeof(float), st));
    CUDA_TRY(cudaMemsetAsync(lp->wb, 0, kBf16Elems * sizeof(__nv_bfloat16), st));
    CUDA_TRY(cudaMemsetAsync(lp->bb, 0, kBiasFloats * sizeof(float), st));
    lp_refresh_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(lp->w, lp->wb, lp->bb);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(st));
    lp->step = 0;
    return FEM_OK;
}

}  // namespace

namespace femi {
// the blocks M_n at u: the block diagonal, then features, network and block
// map in one kernel
fem_status lp_precondition(const void* lpv, fem_mesh* m, const float* u, float* Minv, cudaStream_t st) {
    const fem_lp* lp = static_cast<const fem_lp*>(lpv);
    FEM_TRY(check_lp(lp));
    FEM_TRY(ensure_mesh(m, st));
    LpMeshData* d = m->lp;
    FEM_TRY(run_op(m, FEM_F32, fem::OP_BLOCKDIAG, u, nullptr, d->D, nullptr, 0, st, nullptr));
    lp_pack_kernel<<<grid_for(d->nn, 1184), kVecT, 0, st>>>(d->nn, d->D, d->D8);
    const int64_t groups = (d->nn + 31) / 32;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((groups + 3) / 4, 148 * 5));
    lp_precond_kernel<<<grid, kPrecondThreads, 0, st>>>(d->nn, d->D, d->D8, d->ptr, d->idx, d->stats, m->node_mask,
                                                       InferW{lp->wb, lp->bb}, Minv);
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}
}  // namespace femi

extern "C" {

fem_status fem_lp_create(uint64_t seed, fem_lp** out) {
    if (!out) return fail(FEM_ERR_ARG, "null output pointer");
    *out = nullptr;
    auto* lp = new fem_lp();
    CUDA_TRY(cudaGetDevice(&lp->device));
    void* p = nullptr;
    const size_t bytes = 3 * kParams * sizeof(float) + kBf16Elems * sizeof(__nv_bfloat16) + kBiasFloats * sizeof(float);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        delete lp;
        return fail(FEM_ERR_CUDA, "cudaMalloc of the network parameters failed");
    }
    char* c = static_cast<char*>(p);
    lp->w = reinterpret_cast<float*>(c);
    lp->m = lp->w + kParams;
    lp->v = lp->m + kParams;
    lp->wb = reinterpret_cast<__nv_bfloat16*>(lp->v + kParams);
    lp->bb = reinterpret_cast<float*>(lp->wb + kBf16Elems);
    std::vector<float> w;
    initial_params(seed, w);
    fem_status s = upload_params(lp, w.data(), nullptr);
    if (s != FEM_OK) {
        cudaFree(p);
        delete lp;
        return s;
    }
    *out = lp;
    return FEM_OK;
}

fem_status fem_lp_destroy(fem_lp* lp) {
    if (!lp) return FEM_OK;
    cudaDeviceSynchronize();
    cudaFree(lp->w);
    delete lp;
    return FEM_OK;
}

fem_status fem_lp_set_loss(fem_lp* lp, int kind) {
    FEM_TRY(check_lp(lp));
    if (kind != FEM_LP_LOSS_RESIDUAL && kind != FEM_LP_LOSS_ENERGY) return fail(FEM_ERR_ARG, "unknown loss");
    lp->loss = kind;
    return FEM_OK;
}

fem_status fem_lp_set_clip(fem_lp* lp, float max_grad_norm) {
    FEM_TRY(check_lp(lp));
    if (!(max_grad_norm >= 0.0f)) return fail(FEM_ERR_ARG, "need max_grad_norm >= 0");
    lp->clip = max_grad_norm;
    return FEM_OK;
}

fem_status fem_lp_get_params(const fem_lp* lp, float* params) {
    FEM_TRY(check_lp(lp));
    if (!params) return fail(FEM_ERR_ARG, "null parameter buffer");
    CUDA_TRY(cudaMemcpy(params, lp->w, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    return FEM_OK;
}

fem_status fem_lp_set_params(fem_lp* lp, const float* params) {
    FEM_TRY(check_lp(lp));
    if (!params) return fail(FEM_ERR_ARG, "null parameter buffer");
    return upload_params(lp, params, nullptr);
}

fem_status fem_lp_features(fem_mesh* m, const float* u, void* X, void* stream) {
    if (!m || !u || !X) return fail(FEM_ERR_ARG, "null mesh, u or X");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FEM_TRY(features(m, u, st));
    CUDA_TRY(cudaMemcpyAsync(X, m->lp->X, (size_t)m->lp->nn * kInPad * sizeof(__nv_bfloat16),
                             cudaMemcpyDeviceToDevice, st));
    return FEM_OK;
}

fem_status fem_lp_blocks(const fem_lp* lp, fem_mesh* m, const float* u, float* Minv, void* stream) {
    FEM_TRY(check_lp(lp));
    if (!m || !u || !Minv) return fail(FEM_ERR_ARG, "null mesh, u or Minv");
    return femi::lp_precondition(lp, m, u, Minv, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {
// loss at (u, r) and its weight gradient into m->lp->grad; loss3 on the device
fem_status gradient(fem_lp* lp, fem_mesh* m, const float* u, const float* r, cudaStream_t st, double** loss3_out) {
    FEM_TRY(check_lp(lp));
    if (!m || !u || !r) return fail(FEM_ERR_ARG, "null mesh, u or r");
    FEM_TRY(features(m, u, st));
    femi::LpMeshData* d = m->lp;
    const int64_t nn = d->nn, nd = nn * 3;
    FEM_TRY(infer(lp, m, d->Minv, st));
    lp_apply_kernel<<<grid_for(nn, 1184), kVecT, 0, st>>>(nn, d->Minv, r, d->z);
    // H z, e = H z - r, the loss; then dL/dz = 2 H e / r.r (residual loss)
    // or 2 e / r.r (energy loss)
    FEM_TRY(femi::run_op(m, FEM_F32, fem::OP_HVP, u, d->z, d->q, nullptr, FEM_MASK_BOTH, st, nullptr));
    const int rb = grid_for(nd, kRedBlocks);
    lp_residual_kernel<<<rb, kVecT, 0, st>>>(nd, d->q, r, d->z, d->e, d->red);
    double* loss3 = d->red + (size_t)kRedBlocks * 4;
    lp_loss_kernel<<<1, 32, 0, st>>>(rb, d->red, lp->loss, loss3);
    float* gz = d->e;
    if (lp->loss == FEM_LP_LOSS_RESIDUAL) {
        FEM_TRY(femi::run_op(m, FEM_F32, fem::OP_HVP, u, d->e, d->q, nullptr, FEM_MASK_BOTH, st, nullptr));
        gz = d->q;
    }
    lp_scale_kernel<<<grid_for(nd, 1184), kVecT, 0, st>>>(nd, gz, loss3);
    static bool attr_set = false;
    if (!attr_set) {
        CUDA_TRY(cudaFuncSetAttribute(lp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem)));
        attr_set = true;
    }
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((nn + kGradTile - 1) / kGradTile, kGradBlocks));
    lp_grad_kernel<<<gb, kGradThreads, sizeof(GradSmem), st>>>(nn, d->X, d->D, m->node_mask, r, gz,
                                                               InferW{lp->wb, lp->bb}, d->partial);
    lp_sum_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(gb, d->partial, d->grad);
    CUDA_TRY(cudaGetLastError());
    *loss3_out = loss3;
    return FEM_OK;
}

fem_status read_loss(const double* loss3, double* loss, cudaStream_t st) {
    double h[3];
    CUDA_TRY(cudaMemcpyAsync(h, loss3, sizeof h, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    *loss = h[2];
    return FEM_OK;
}
}  // namespace

extern "C" {

fem_status fem_lp_gradient(fem_lp* lp, fem_mesh* m, const float* u, const float* r, float* grad, double* loss,
                           void* stream) {
    if (!grad) return fail(FEM_ERR_ARG, "null gradient buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* loss3 = nullptr;
    FEM_TRY(gradient(lp, m, u, r, st, &loss3));
    CUDA_TRY(cudaMemcpyAsync(grad, m->lp->grad, kParams * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (loss) return read_loss(loss3, loss, st);
    CUDA_TRY(cudaStreamSynchronize(st));
    return FEM_OK;
}

fem_status fem_lp_train_step(fem_lp* lp, fem_mesh* m, const float* u, const float* r, float lr, double* loss,
                             void* stream) {
    if (!(lr > 0.0f)) return fail(FEM_ERR_ARG, "need lr > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* loss3 = nullptr;
    FEM_TRY(gradient(lp, m, u, r, st, &loss3));
    ++lp->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)lp->step), c2 = 1.0f - std::pow(b2, (float)lp->step);
    float* scale = m->lp->grad + kParams;
    lp_clip_kernel<<<1, kVecT, 0, st>>>(m->lp->grad, lp->clip, scale);
    lp_adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(m->lp->grad, scale, lp->w, lp->m, lp->v, lr, b1, b2, 1e-8f,
                                                          c1, c2, lp->wb, lp->bb);
    CUDA_TRY(cudaGetLastError());
    if (loss) return read_loss(loss3, loss, st);
    return FEM_OK;
}

}  // extern "C"
