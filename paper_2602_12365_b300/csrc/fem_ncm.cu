// Neural constitutive model (Sec. "Neural Constitutive Modeling"):
//   psi = [NN(I1, J) - NN(3, 1)] + psi_NH(mu_e, lambda_e),
// NN a 2 -> H -> H -> 1 MLP with softplus activations of the invariants
// I1 = tr(F^T F) (+1 in plane strain) and J = det F, shared by all elements.
//
// The network enters the element operators only through its value, gradient
// and Hessian in (I1, J) at each element.  Those are computed for all
// elements by one pass of the tile kernel (OP_NCM_INV: each element's
// I1 - 3 and J - 1, in record order) and the network kernel below (one thread
// per element: forward pass, gradient and Hessian), and the element kernels
// read them as eight coefficients per element.  In a PCG solve the state is
// fixed, so the solver evaluates the network once per solve.
//
// Network kernel: with a1 = sp(z1), s1 = s(z1) (s the logistic sigmoid, the
// derivative of softplus), z2_m = b2_m + W2_m . a1 and the tangents
// u_m^j = sum_k W2[m][k] s1_k W1[k][j] of z2_m along the inputs j:
//   dNN/dx_j = sum_m w3_m s(z2_m) u_m^j,
//   d2NN/dx_i dx_j = sum_m w3_m s'(z2_m) u_m^i u_m^j
//                  + sum_k (sum_m W2[m][k] w3_m s(z2_m)) s'(z1_k) W1[k][i] W1[k][j],
// the last sum accumulated in one vector over the units k, so the kernel
// keeps three H-vectors per thread and does 4 H^2 multiply-adds.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fem_b300.h"
#include "fem_internal.h"

namespace femi {
struct NcmData {
    int H = 0;
    double nn0 = 0.0;                     // NN(3, 1)
    std::vector<double> host;             // parameters (kernel arguments)
    void* inv[2] = {nullptr, nullptr};    // [n_rec][2] per precision (FP64, FP32)
    void* coef[2] = {nullptr, nullptr};   // [n_rec][8]
    int64_t n_rec = 0;
    std::vector<void*> allocs;
};

void ncm_free(fem_mesh* m) {
    if (!m || !m->ncm) return;
    for (void* p : m->ncm->allocs) cudaFree(p);
    delete m->ncm;
    m->ncm = nullptr;
}

const void* ncm_coef(const fem_mesh* m, int pi) { return m->ncm ? m->ncm->coef[pi] : nullptr; }
void* ncm_inv(const fem_mesh* m, int pi) { return m->ncm ? m->ncm->inv[pi] : nullptr; }
}  // namespace femi

namespace {

constexpr int kT = 256;

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

__host__ __device__ constexpr int n_params(int H) { return H * H + 5 * H + 1; }

// NN(I1, J) on the host in FP64 (the shift NN(3, 1))
double host_nn(int H, const double* p, double I1, double J) {
    const double *W1 = p, *b1 = W1 + 2 * H, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H;
    auto sp = [](double t) { return t > 30.0 ? t : std::log1p(std::exp(t)); };
    std::vector<double> a1(H);
    for (int k = 0; k < H; ++k) a1[k] = sp(W1[2 * k] * I1 + W1[2 * k + 1] * J + b1[k]);
    double y = w3[H];
    for (int m = 0; m < H; ++m) {
        double z = b2[m];
        for (int k = 0; k < H; ++k) z += W2[m * H + k] * a1[k];
        y += w3[m] * sp(z);
    }
    return y;
}

// FP32: the hardware exp2/log2 intrinsics (a few ulp; the coefficients enter
// the operators at the ~1e-6 level, inside the FP32 bar), FP64: exact
// functions.  softplus(t) = ln(1 + e^t) is taken as t beyond 20 (30 in FP64),
// where the two agree to rounding.
__device__ __forceinline__ float softplus_(float t) { return t > 20.f ? t : __logf(1.f + __expf(t)); }
__device__ __forceinline__ double softplus_(double t) { return t > 30.0 ? t : log1p(exp(t)); }
__device__ __forceinline__ float sigmoid_(float t) { return __fdividef(1.f, 1.f + __expf(-t)); }
__device__ __forceinline__ double sigmoid_(double t) { return 1.0 / (1.0 + exp(-t)); }
// softplus and its derivative (the sigmoid) from one exponential: with
// e = exp(t), softplus = log1p(e) and sigmoid = e / (1 + e); above the
// softplus cut-off, softplus = t and the sigmoid keeps its own form
__device__ __forceinline__ void softplus_sigmoid_(float t, float& sp, float& sg) {
    if (t > 20.f) {
        sp = t;
        sg = sigmoid_(t);
    } else {
        const float e = __expf(t);
        sp = __logf(1.f + e);
        sg = __fdividef(e, 1.f + e);
    }
}
__device__ __forceinline__ void softplus_sigmoid_(double t, double& sp, double& sg) {
    if (t > 30.0) {
        sp = t;
        sg = sigmoid_(t);
    } else {
        const double e = exp(t);
        sp = log1p(e);
        sg = e / (1.0 + e);
    }
}

template <typename T>
__device__ __forceinline__ void store8(T* dst, const T (&c)[8]) {
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(c[0], c[1], c[2], c[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(c[4], c[5], c[6], c[7]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) reinterpret_cast<double2*>(dst)[j] = make_double2(c[2 * j], c[2 * j + 1]);
    }
}

// the network's parameters as one kernel argument: every multiply-add takes
// its weight from the parameter constant bank at a compile-time offset (no
// load instruction); H = 32 in FP64 is 9,480 bytes, within the argument limit
template <typename T, int H>
struct NcmArgs {
    T w[H * H + 5 * H + 1];
};

// coefficients per element, as much as `MODE` needs: 0 (energy) the value
// NN - NN(3, 1) and its roundoff scale |NN| + |NN(3, 1)|; 1 (residual) also
// dNN/dI1, dNN/dJ; 2 (HVP, block diagonal) also d2NN/dI1^2, d2NN/dI1 dJ,
// d2NN/dJ^2.  The gradient by reverse accumulation over the units k
// (back_k = sum_m W2[m][k] w3_m s(z2_m)); the Hessian as in the file comment.
template <typename T, int H, int MODE>
__global__ void __launch_bounds__(kT) ncm_coef_kernel(int64_t n, const T* __restrict__ inv, const NcmArgs<T, H> prm,
                                                      T nn0, T* __restrict__ coef, const int* skip) {
    if (skip != nullptr && *skip != 0) return;
    const T *W1 = prm.w, *b1 = W1 + 2 * H, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H;
    for (int64_t e = blockIdx.x * (int64_t)kT + threadIdx.x; e < n; e += (int64_t)gridDim.x * kT) {
        const T I1 = T(3) + inv[2 * e], J = T(1) + inv[2 * e + 1];
        T a1[H], s1[H], back[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const T z = W1[2 * k] * I1 + W1[2 * k + 1] * J + b1[k];
            if constexpr (MODE >= 1)
                softplus_sigmoid_(z, a1[k], s1[k]);
            else
                a1[k] = softplus_(z);
            back[k] = T(0);
        }
        T y = w3[H], h00 = T(0), h01 = T(0), h11 = T(0);
#pragma unroll
        for (int m = 0; m < H; ++m) {
            T z2 = b2[m];
#pragma unroll
            for (int k = 0; k < H; ++k) z2 += W2[m * H + k] * a1[k];
            T sp2, s2 = T(0);
            if constexpr (MODE >= 1)
                softplus_sigmoid_(z2, sp2, s2);
            else
                sp2 = softplus_(z2);
            y += w3[m] * sp2;
            if constexpr (MODE >= 1) {
                const T gm = w3[m] * s2;
#pragma unroll
                for (int k = 0; k < H; ++k) back[k] += W2[m * H + k] * gm;
                if constexpr (MODE == 2) {
                    T u0 = T(0), u1 = T(0);
#pragma unroll
                    for (int k = 0; k < H; ++k) {
                        const T ws = W2[m * H + k] * s1[k];
                        u0 += ws * W1[2 * k];
                        u1 += ws * W1[2 * k + 1];
                    }
                    const T ht = gm * (T(1) - s2);
                    h00 += ht * u0 * u0;
                    h01 += ht * u0 * u1;
                    h11 += ht * u1 * u1;
                }
            }
        }
        T c[8] = {y - nn0, fabs(y) + fabs(nn0), T(0), T(0), T(0), T(0), T(0), T(0)};
        if constexpr (MODE >= 1) {
            T g0 = T(0), g1 = T(0);
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const T bs = back[k] * s1[k];
                g0 += bs * W1[2 * k];
                g1 += bs * W1[2 * k + 1];
                if constexpr (MODE == 2) {
                    const T bt = bs * (T(1) - s1[k]);
                    h00 += bt * W1[2 * k] * W1[2 * k];
                    h01 += bt * W1[2 * k] * W1[2 * k + 1];
                    h11 += bt * W1[2 * k + 1] * W1[2 * k + 1];
                }
            }
            c[2] = g0, c[3] = g1, c[4] = h00, c[5] = h01, c[6] = h11;
        }
        store8(coef + e * 8, c);
    }
}

template <typename T, int H>
fem_status run_h(const femi::NcmData* N, int pi, int mode, cudaStream_t st, const int* skip) {
    NcmArgs<T, H> a;
    const std::vector<double>& hp = N->host;
    for (int i = 0; i < n_params(H); ++i) a.w[i] = (T)hp[i];
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N->n_rec + kT - 1) / kT, 148 * 8));
    const T* inv = static_cast<const T*>(N->inv[pi]);
    T* coef = static_cast<T*>(N->coef[pi]);
    const T nn0 = (T)N->nn0;
    if (mode == 0)
        ncm_coef_kernel<T, H, 0><<<grid, kT, 0, st>>>(N->n_rec, inv, a, nn0, coef, skip);
    else if (mode == 1)
        ncm_coef_kernel<T, H, 1><<<grid, kT, 0, st>>>(N->n_rec, inv, a, nn0, coef, skip);
    else
        ncm_coef_kernel<T, H, 2><<<grid, kT, 0, st>>>(N->n_rec, inv, a, nn0, coef, skip);
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

// ---------------------------------------------------------------------------
// FP32 network on the tensor cores (H = 16, 32).  A warp takes 16 elements
// (rows).  The three H x H products -- z2 = a1 W2^T, back = G W2 with
// G_m = w3_m s(z2_m), and the tangents u_j = (s1 * W1[:, j]) W2^T -- run as
// mma.sync m16n8k16 with FP16 operands and FP32 accumulation.  Each FP32
// operand x is split into FP16 parts x = x_hi + x_lo (x_lo the rounded rest)
// and a product is taken as a_hi b_hi + a_lo b_hi + a_hi b_lo, the split-
// precision scheme of Markidis et al. (2018) and Ootomo & Yokota (2022): the
// dropped a_lo b_lo and the rounding of the parts leave about 2^-22 relative,
// FP32 accuracy, which plain FP16/BF16 (2^-11, 2^-8) would not give.
//
// Per lane, a row-by-column block is held in the accumulator layout of
// m16n8: X[j][0..3] = (row g, col 8j+2t), (g, 8j+2t+1), (g+8, 8j+2t),
// (g+8, 8j+2t+1) with g = lane / 4, t = lane % 4; the accumulators of column
// tiles 2kk and 2kk+1 are, element for element, the A fragment of K chunk kk
// of the next product.  Per-row sums over the columns end with a butterfly
// over the four lanes of a row.
// ---------------------------------------------------------------------------
constexpr int kTcThreads = 128;

struct HalfPair {
    uint32_t hi, lo;
};

__device__ __forceinline__ HalfPair split2(float a, float b) {
    const __half ah = __float2half_rn(a), bh = __float2half_rn(b);
    const __half al = __float2half_rn(a - __half2float(ah)), bl = __float2half_rn(b - __half2float(bh));
    const __half2 h = __halves2half2(ah, bh), l = __halves2half2(al, bl);
    return HalfPair{*reinterpret_cast<const uint32_t*>(&h), *reinterpret_cast<const uint32_t*>(&l)};
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// D[j] += A B over K = H: A in the accumulator layout (FP32, split here), B
// as FP16 hi/lo rows of length H (row n of B^T: b(k, n) = Bt[n][k]), stride S
template <int H, int S>
__device__ __forceinline__ void tc_gemm(float (&D)[H / 8][4], const float (&A)[H / 8][4], const __half* Bh,
                                        const __half* Bl, int g, int t) {
#pragma unroll
    for (int kk = 0; kk < H / 16; ++kk) {
        uint32_t ah[4], al[4];
        const HalfPair p0 = split2(A[2 * kk][0], A[2 * kk][1]);
        const HalfPair p1 = split2(A[2 * kk][2], A[2 * kk][3]);
        const HalfPair p2 = split2(A[2 * kk + 1][0], A[2 * kk + 1][1]);
        const HalfPair p3 = split2(A[2 * kk + 1][2], A[2 * kk + 1][3]);
        ah[0] = p0.hi, ah[1] = p1.hi, ah[2] = p2.hi, ah[3] = p3.hi;
        al[0] = p0.lo, al[1] = p1.lo, al[2] = p2.lo, al[3] = p3.lo;
#pragma unroll
        for (int j = 0; j < H / 8; ++j) {
            const int o = (8 * j + g) * S + 16 * kk + 2 * t;
            const uint32_t bh0 = *reinterpret_cast<const uint32_t*>(Bh + o);
            const uint32_t bh1 = *reinterpret_cast<const uint32_t*>(Bh + o + 8);
            const uint32_t bl0 = *reinterpret_cast<const uint32_t*>(Bl + o);
            const uint32_t bl1 = *reinterpret_cast<const uint32_t*>(Bl + o + 8);
            mma_f16(D[j], ah, bh0, bh1);
            mma_f16(D[j], al, bh0, bh1);
            mma_f16(D[j], ah, bl0, bl1);
        }
    }
}

__device__ __forceinline__ float quad_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

template <int H, int MODE>
__global__ void __launch_bounds__(kTcThreads) ncm_coef_tc_kernel(int64_t n, const float* __restrict__ inv,
                                                                 const NcmArgs<float, H> prm, float nn0,
                                                                 float* __restrict__ coef, const int* skip) {
    constexpr int S = H + 8;  // row stride in halves (conflict-free fragment loads)
    __shared__ __align__(16) __half sW2h[H * S], sW2l[H * S], sWTh[H * S], sWTl[H * S];
    if (skip != nullptr && *skip != 0) return;
    const float *W1 = prm.w, *b1 = W1 + 2 * H, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H;
    for (int i = threadIdx.x; i < H * H; i += kTcThreads) {
        const int m = i / H, k = i % H;
        const float w = W2[i];
        const __half h = __float2half_rn(w), l = __float2half_rn(w - __half2float(h));
        sW2h[m * S + k] = h, sW2l[m * S + k] = l;  // W2 as rows m
        sWTh[k * S + m] = h, sWTl[k * S + m] = l;  // W2^T as rows k
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t n_tiles = (n + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * (kTcThreads / 32) + warp; tile < n_tiles;
         tile += (int64_t)gridDim.x * (kTcThreads / 32)) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        const float I10 = r0 < n ? 3.f + inv[2 * r0] : 3.f, J0 = r0 < n ? 1.f + inv[2 * r0 + 1] : 1.f;
        const float I11 = r1 < n ? 3.f + inv[2 * r1] : 3.f, J1 = r1 < n ? 1.f + inv[2 * r1 + 1] : 1.f;
        // layer 1 on the CUDA cores, in the accumulator layout
        float a1[H / 8][4], s1[H / 8][4], z2[H / 8][4];
#pragma unroll
        for (int j = 0; j < H / 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 8 * j + 2 * t + (q & 1);
                const float z = W1[2 * c] * (q < 2 ? I10 : I11) + W1[2 * c + 1] * (q < 2 ? J0 : J1) + b1[c];
                a1[j][q] = softplus_(z);
                s1[j][q] = sigmoid_(z);
                z2[j][q] = b2[c];
            }
        tc_gemm<H, S>(z2, a1, sW2h, sW2l, g, t);
        // the value, and G = w3 s(z2) for the gradient
        float y0 = 0.f, y1 = 0.f, G[H / 8][4], s2[H / 8][4];
#pragma unroll
        for (int j = 0; j < H / 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 8 * j + 2 * t + (q & 1);
                const float v = w3[c] * softplus_(z2[j][q]);
                if (q < 2) y0 += v; else y1 += v;
                s2[j][q] = sigmoid_(z2[j][q]);
                G[j][q] = w3[c] * s2[j][q];
            }
        y0 = quad_sum(y0) + w3[H];
        y1 = quad_sum(y1) + w3[H];
        float c0[8] = {y0 - nn0, fabsf(y0) + fabsf(nn0), 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float c1[8] = {y1 - nn0, fabsf(y1) + fabsf(nn0), 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if constexpr (MODE >= 1) {
            float back[H / 8][4];
#pragma unroll
            for (int j = 0; j < H / 8; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) back[j][q] = 0.f;
            tc_gemm<H, S>(back, G, sWTh, sWTl, g, t);
            // gradient sum_k back_k s1_k W1[k][.]; Hessian part sum_k back_k s'(z1_k) W1 W1
            float p[2][5] = {};
#pragma unroll
            for (int j = 0; j < H / 8; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = 8 * j + 2 * t + (q & 1);
                    const float bs = back[j][q] * s1[j][q];
                    const float w0 = W1[2 * c], w1 = W1[2 * c + 1];
                    float* pr = p[q < 2 ? 0 : 1];
                    pr[0] += bs * w0;
                    pr[1] += bs * w1;
                    if constexpr (MODE == 2) {
                        const float bt = bs * (1.f - s1[j][q]);
                        pr[2] += bt * w0 * w0;
                        pr[3] += bt * w0 * w1;
                        pr[4] += bt * w1 * w1;
                    }
                }
            if constexpr (MODE == 2) {
                // tangents of z2 along I1 and J, then sum_m w3 s'(z2_m) u_m^i u_m^j
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    float A[H / 8][4], U[H / 8][4];
#pragma unroll
                    for (int j = 0; j < H / 8; ++j)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            A[j][q] = s1[j][q] * W1[2 * (8 * j + 2 * t + (q & 1)) + jj];
                            U[j][q] = 0.f;
                        }
                    tc_gemm<H, S>(U, A, sW2h, sW2l, g, t);
#pragma unroll
                    for (int j = 0; j < H / 8; ++j)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float ht = G[j][q] * (1.f - s2[j][q]);
                            float* pr = p[q < 2 ? 0 : 1];
                            if (jj == 0) {
                                pr[2] += ht * U[j][q] * U[j][q];
                                z2[j][q] = U[j][q];  // z2 is free now: hold u^0
                            } else {
                                pr[3] += ht * z2[j][q] * U[j][q];
                                pr[4] += ht * U[j][q] * U[j][q];
                            }
                        }
                }
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                p[0][k] = quad_sum(p[0][k]);
                p[1][k] = quad_sum(p[1][k]);
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) c0[2 + k] = p[0][k], c1[2 + k] = p[1][k];
        }
        if (t == 0) {
            if (r0 < n) store8(coef + r0 * 8, c0);
            if (r1 < n) store8(coef + r1 * 8, c1);
        }
    }
}

template <int H>
fem_status run_tc(const femi::NcmData* N, int mode, cudaStream_t st, const int* skip) {
    NcmArgs<float, H> a;
    for (int i = 0; i < n_params(H); ++i) a.w[i] = (float)N->host[i];
    const int64_t tiles = (N->n_rec + 15) / 16;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 3) / 4, 148 * 16));
    const float* inv = static_cast<const float*>(N->inv[1]);
    float* coef = static_cast<float*>(N->coef[1]);
    const float nn0 = (float)N->nn0;
    if (mode == 0)
        ncm_coef_tc_kernel<H, 0><<<grid, kTcThreads, 0, st>>>(N->n_rec, inv, a, nn0, coef, skip);
    else if (mode == 1)
        ncm_coef_tc_kernel<H, 1><<<grid, kTcThreads, 0, st>>>(N->n_rec, inv, a, nn0, coef, skip);
    else
        ncm_coef_tc_kernel<H, 2><<<grid, kTcThreads, 0, st>>>(N->n_rec, inv, a, nn0, coef, skip);
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

template <typename T>
fem_status run_coef(const femi::NcmData* N, int pi, int mode, cudaStream_t st, const int* skip) {
    if constexpr (sizeof(T) == 4) {  // FP32: the tensor cores where H is a multiple of 16
        if (N->H == 16) return run_tc<16>(N, mode, st, skip);
        if (N->H == 32) return run_tc<32>(N, mode, st, skip);
    }
    switch (N->H) {
        case 8: return run_h<T, 8>(N, pi, mode, st, skip);
        case 16: return run_h<T, 16>(N, pi, mode, st, skip);
        default: return run_h<T, 32>(N, pi, mode, st, skip);
    }
}

// device arrays of one precision: parameters are uploaded by the caller;
// the invariants start at zero, so lanes without an element keep the rest
// state (I1, J) = (3, 1)
fem_status alloc_arrays(femi::NcmData* N, int pi) {
    const size_t es = pi == 0 ? sizeof(double) : sizeof(float);
    void *inv = nullptr, *coef = nullptr;
    CUDA_TRY(cudaMalloc(&inv, (size_t)N->n_rec * 2 * es));
    N->allocs.push_back(inv);
    CUDA_TRY(cudaMalloc(&coef, (size_t)N->n_rec * 8 * es));
    N->allocs.push_back(coef);
    CUDA_TRY(cudaMemset(inv, 0, (size_t)N->n_rec * 2 * es));
    N->inv[pi] = inv;
    N->coef[pi] = coef;
    return FEM_OK;
}

fem_status build(fem_mesh* m, int hidden, const double* params, femi::NcmData* N) {
    N->H = hidden;
    N->nn0 = host_nn(hidden, params, 3.0, 1.0);
    N->n_rec = m->plan.n_rounds() * 32;
    N->host.assign(params, params + n_params(hidden));
    FEM_TRY(alloc_arrays(N, 0));
    if (m->precision == FEM_PREC_MIXED) FEM_TRY(alloc_arrays(N, 1));
    return FEM_OK;
}

}  // namespace

namespace femi {
fem_status ncm_prepare(fem_mesh* m, int dtype, cudaStream_t) {
    const int pi = dtype == FEM_F64 ? 0 : 1;
    if (!m->ncm || !m->ncm->inv[pi]) return fail(FEM_ERR_ARG, "neural constitutive model arrays missing");
    return FEM_OK;
}

fem_status ncm_coefficients(fem_mesh* m, int dtype, int mode, cudaStream_t st, const int* skip) {
    return dtype == FEM_F64 ? run_coef<double>(m->ncm, 0, mode, st, skip)
                            : run_coef<float>(m->ncm, 1, mode, st, skip);
}
}  // namespace femi

extern "C" {

fem_status fem_mesh_set_ncm(fem_mesh* m, int hidden, const double* params) {
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    if (hidden == 0) {
        cudaDeviceSynchronize();  // kernels in flight may still read the old arrays
        femi::ncm_free(m);
        return FEM_OK;
    }
    if (hidden != 8 && hidden != 16 && hidden != 32) return fail(FEM_ERR_ARG, "hidden must be 0, 8, 16 or 32");
    if (!params) return fail(FEM_ERR_ARG, "null params");
    if (m->etype == FEM_HEX8) return fail(FEM_ERR_ARG, "the neural constitutive model covers P1 elements");
    for (int i = 0; i < n_params(hidden); ++i)
        if (!std::isfinite(params[i])) return fail(FEM_ERR_NONFINITE, "non-finite network parameter");
    auto* N = new femi::NcmData();
    const fem_status s = build(m, hidden, params, N);
    if (s != FEM_OK) {
        for (void* p : N->allocs) cudaFree(p);
        delete N;
        return s;
    }
    cudaDeviceSynchronize();  // kernels in flight may still read the old arrays
    femi::ncm_free(m);
    m->ncm = N;
    return FEM_OK;
}

}  // extern "C"
