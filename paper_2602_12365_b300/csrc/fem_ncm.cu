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
            a1[k] = softplus_(z);
            if constexpr (MODE >= 1) s1[k] = sigmoid_(z);
            back[k] = T(0);
        }
        T y = w3[H], h00 = T(0), h01 = T(0), h11 = T(0);
#pragma unroll
        for (int m = 0; m < H; ++m) {
            T z2 = b2[m];
#pragma unroll
            for (int k = 0; k < H; ++k) z2 += W2[m * H + k] * a1[k];
            y += w3[m] * softplus_(z2);
            if constexpr (MODE >= 1) {
                const T s2 = sigmoid_(z2);
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

template <typename T>
fem_status run_coef(const femi::NcmData* N, int pi, int mode, cudaStream_t st, const int* skip) {
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
