// Matrix-free Newton-CG load step on the device (fem_newton_step).
//
// The paper minimises the total potential with Newton-Krylov iterations
// built on the residual and its directional derivative (Sec. 6.3.1, 6.6) and
// leaves the details open; this driver fixes one algorithm, step for step
// the same as the oracle's load step:
//   1. du_c = (s - s_prev) ubar on prescribed DOFs.
//   2. predictor t = M K(u) (I - M) du_c, r0 = ||t||; PCG on M K M du_f = -t
//      to relative tolerance 1e-2; u += du_c + du_f; prescribed u = s ubar.
//   3. Newton: r = M grad Psi(u); stop when ||r|| <= rtol r0; PCG on
//      M K M d = -r from 0 to eta ||r||, eta = min(eta_max, sqrt(||r||/r0))
//      (non-positive curvature: first iteration d = P r, later the current
//      iterate); backtracking Armijo on Psi with the roundoff guard
//      |dPsi| <= 16 eps S and ||r|| decreasing; u += alpha d.
//   4. an inverted predictor, a failed line search, a non-SPD block or
//      newton_max iterations restore u and bisect the increment.
// The preconditioner is block Jacobi: each nodal diagonal block inverted
// through its Cholesky factor.
//
// Precision: u, the Newton residual and the line-search energies are FP64
// in every mode (a converged residual of 1e-8 r0 and energy differences near
// the roundoff floor need it).  cg_dtype FEM_F32 runs the PCG -- its HVPs,
// block diagonal, preconditioner and vectors -- in FP32 on an FP32 shadow of
// u, with every dot product and norm accumulated in FP64.
//
// The PCG loop runs on the device, in the Chronopoulos-Gear form (one HVP
// with its fused z . K z and one update kernel per iteration; the iterates
// are those of standard PCG): alpha, beta, the residual norm and a `done`
// state live in device memory, every kernel of an iteration returns at once
// when done is set, and the host enqueues iterations in batches and
// reads done one batch behind, so the GPU never waits for the host inside a
// solve.  Every reduction is a fixed-order FP64 sum (per-thread strided
// sums, a warp butterfly, warps in order, blocks in order by the last block),
// so results are bitwise reproducible for a given mesh and device.
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

constexpr int kVT = 256;          // threads of the vector kernels
constexpr int kMaxRedBlocks = 1184;  // partial-sum slots (8 blocks per SM on 148 SMs)
constexpr int kVecBlocks = 592;      // grid of the vector kernels: 4 blocks per SM

// device-resident scalars of one PCG solve (Chronopoulos-Gear form)
struct CgState {
    double rgamma[2];  // 1 / (r . z) of launch k in slot k & 1 (read by launch k + 1)
    double pkp[2];     // p^T K p of launch k in slot k & 1
    double rr;         // r . r at the stop
    double tol2;       // squared absolute tolerance on ||r||
    long long cg_max;
    int done;  // 0 running, 1 converged, 2 non-positive curvature, 3 iteration cap
    int k;     // iterations (HVPs) performed, set at the stop
};

struct DotState {
    double value;
    unsigned counter;
    int pad;
};

// ---------------------------------------------------------------------------
// Dot-product accumulators.  FP64 vectors add in double.  FP32 vectors keep
// an unevaluated float pair hi + lo: each product a*b is split exactly into
// p + e by an FMA (e = fma(a, b, -p)) and added with Knuth's TwoSum, so the
// pair carries the sum to about 2^-44 relative; it is widened to double once
// per warp.  On this GPU FP64 instructions issue at a small fraction of the
// FP32 rate, and these sums run in every CG iteration.
// ---------------------------------------------------------------------------
struct FF {
    float hi = 0.f, lo = 0.f;
};

__device__ __forceinline__ void ff_add(FF& s, float x) {
    const float t = s.hi + x;
    const float bp = t - s.hi;
    s.lo += (s.hi - (t - bp)) + (x - bp);
    s.hi = t;
}
__device__ __forceinline__ void acc_prod(FF& s, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    ff_add(s, p);
    s.lo += e;
}
__device__ __forceinline__ void acc_prod(double& s, double a, double b) { s = fma(a, b, s); }

template <typename T>
struct AccT {
    using type = double;
};
template <>
struct AccT<float> {
    using type = FF;
};

// warp butterfly on the accumulator (all lanes end with the warp's sum);
// FP32 pairs stay pairs, widened to double by the one lane that stores them
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ FF warp_sum(FF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, v.hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, v.lo, o);
        ff_add(v, oh);
        v.lo += ol;
    }
    return v;
}
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(FF v) { return (double)v.hi + (double)v.lo; }

// ---------------------------------------------------------------------------
// fixed-order block reduction of NV doubles; the total lands in thread 0
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_total(double (&v)[NV], double* sh /* [kVT/32 * NV] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kVT / 32; ++w)
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] += sh[w * NV + k];
}

// Each block stores its partial sums; the last block to arrive adds the
// partials in block order and returns true (its thread 0 holds the totals).
// A: double, or FF (FP32 pairs, widened per warp).
template <int NV, typename A>
__device__ __forceinline__ bool grid_total(A (&a)[NV], double (&out)[NV], double* partial, unsigned* counter) {
    __shared__ double sh[kVT / 32 * NV];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] = warp_sum(a[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp * NV + k] = v[k] = widen(a[k]);
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kVT / 32; ++w)
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] += sh[w * NV + k];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[blockIdx.x * NV + k] = v[k];
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1u);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double t[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kVT)
#pragma unroll
        for (int k = 0; k < NV; ++k) t[k] += __ldcg(partial + b * NV + k);
    block_total<NV>(t, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = t[k];
        *counter = 0u;
    }
    return true;
}

// z = Minv_n r for one node (D x D row-major block)
template <int D, typename T>
__device__ __forceinline__ void apply_block(const T* Minv, int64_t n, const T (&r)[3], T (&z)[3]) {
    const T* M = Minv + n * D * D;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T s = M[i * D] * r[0];
#pragma unroll
        for (int j = 1; j < D; ++j) s += M[i * D + j] * r[j];
        z[i] = s;
    }
}

// 16-byte vector access to E contiguous values (E * sizeof(T) a multiple of
// 16, the address 16-byte aligned)
template <typename T, int E>
__device__ __forceinline__ void ld16(const T* src, T (&v)[E]) {
    static_assert((E * sizeof(T)) % 16 == 0, "whole 16-byte chunks");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < E / 4; ++k) {
            const float4 q = reinterpret_cast<const float4*>(src)[k];
            v[4 * k] = q.x, v[4 * k + 1] = q.y, v[4 * k + 2] = q.z, v[4 * k + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < E / 2; ++k) {
            const double2 q = reinterpret_cast<const double2*>(src)[k];
            v[2 * k] = q.x, v[2 * k + 1] = q.y;
        }
    }
}
template <typename T, int E>
__device__ __forceinline__ void st16(T* dst, const T (&v)[E]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < E / 4; ++k)
            reinterpret_cast<float4*>(dst)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < E / 2; ++k) reinterpret_cast<double2*>(dst)[k] = make_double2(v[2 * k], v[2 * k + 1]);
    }
}
// nodes per group so that a group's values of one vector are whole 16-byte
// chunks (3D FP32: 4 nodes = 48 bytes)
__host__ __device__ constexpr int node_group(int D, int tsize) {
    return (D * tsize) % 16 == 0 ? 1 : ((D * tsize) % 8 == 0 ? 2 : 4);
}

// ---------------------------------------------------------------------------
// PCG kernels
// ---------------------------------------------------------------------------
// PCG in the Chronopoulos-Gear form: the iterates of the standard
// preconditioned CG (x_k, r_k, p_k, one HVP per iteration, the same stop and
// non-positive-curvature rules), with s = K p carried by recurrence so that an
// iteration needs one HVP, w = K z (its z . K z fused into the HVP), and one
// update kernel:
//   beta = gamma / gamma_old, p^T K p = delta - beta gamma / alpha_old,
//   alpha = gamma / p^T K p, p = z + beta p, s = w + beta s,
//   x += alpha p, r -= alpha s, z = M r.
// No kernel waits for a grid-wide sum.  Each update kernel leaves per-block
// partial sums of r . r and r . z (slot (k + 1) & 1 of the partial buffer);
// the next one (launch k + 1, after the HVP) has every block add those and
// the HVP's per-tile z . K z partials in the same fixed order, so every
// block holds the same gamma, delta and ||r|| and takes the same decision:
// stop (converged, iteration cap, non-positive curvature) or update.  The
// stop is therefore seen one launch after the update that reached it, and
// that launch's HVP is the only work spent past the stop.  cg_init and every
// cg_step of one solve run on the same grid (the partial count).

// accumulator + accumulator (pair or double)
__device__ __forceinline__ void acc_add(FF& s, FF x) {
    ff_add(s, x.hi);
    s.lo += x.lo;
}
__device__ __forceinline__ void acc_add(double& s, double x) { s += x; }
// L2 load of an accumulator another kernel wrote
__device__ __forceinline__ FF ld_acc(const FF* q) {
    const float2 x = __ldcg(reinterpret_cast<const float2*>(q));
    FF f;
    f.hi = x.x;
    f.lo = x.y;
    return f;
}
__device__ __forceinline__ double ld_acc(const double* q) { return __ldcg(q); }

// fixed-order block sum of NV accumulators; the totals land in thread 0
template <int NV, typename A>
__device__ __forceinline__ void block_sum(A (&a)[NV], A* sh /* [kVT / 32 * NV] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] = warp_sum(a[k]);
    __syncthreads();  // sh may hold an earlier sum
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp * NV + k] = a[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kVT / 32; ++w)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc_add(a[k], sh[w * NV + k]);
}

// r = b, z = M b, x = p = s = 0; per-block r . r and r . z into slot 0
template <int D, typename T>
__global__ void __launch_bounds__(kVT) cg_init(int64_t nn, const T* b, T* x, T* r, T* z, T* p, T* s,
                                               const T* Minv, CgState* st,
                                               typename AccT<T>::type* partial) {
    using A = typename AccT<T>::type;
    __shared__ A sh[kVT / 32 * 2];
    A v[2] = {};
    for (int64_t n = blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
        T rv[3] = {0, 0, 0}, zz[3];
#pragma unroll
        for (int c = 0; c < D; ++c) rv[c] = b[n * D + c];
        apply_block<D, T>(Minv, n, rv, zz);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            x[n * D + c] = T(0);
            r[n * D + c] = rv[c];
            z[n * D + c] = zz[c];
            p[n * D + c] = T(0);
            s[n * D + c] = T(0);
            acc_prod(v[0], rv[c], rv[c]);
            acc_prod(v[1], rv[c], zz[c]);
        }
    }
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = v[0];
        partial[2 * blockIdx.x + 1] = v[1];
        if (blockIdx.x == 0) {
            st->done = 0;
            st->k = 0;
        }
    }
}

// one partial of z . K z per HVP tile (an FP32 pair, or a double)
template <typename T>
__device__ __forceinline__ typename AccT<T>::type tile_partial(const double* tile_red, int t) {
    if constexpr (sizeof(T) == 4) {
        const float2 x = __ldcg(reinterpret_cast<const float2*>(tile_red + (int64_t)t * 4));
        FF f;
        f.hi = x.x;
        f.lo = x.y;
        return f;
    } else {
        return __ldcg(tile_red + (int64_t)t * 4);
    }
}

// launch k of a solve (k = 0, 1, ... counted by the host)
template <int D, typename T>
__global__ void __launch_bounds__(kVT) cg_step(int64_t nn, long long k, T* x, T* r, T* z, T* p, T* s, const T* w,
                                               const T* Minv, CgState* st, typename AccT<T>::type* partial,
                                               const double* tile_red, int n_tiles) {
    using A = typename AccT<T>::type;
    // Launched as a programmatic dependent launch of the HVP's finalize
    // kernel.  Its blocks start only once every finalize block has exited, and
    // each of those first waited for the HVP's tile kernel, which itself
    // waited for the previous update kernel (or cg_init) to complete.  So
    // what that update kernel wrote (x, r, z, p, s, the block partials, the
    // state) is visible from the start; w and the tile partials only after
    // griddepcontrol.wait.
    if (st->done) return;  // a stop taken by an earlier launch (or by this one: same decision)
    __shared__ A sh[kVT / 32 * 3];
    __shared__ T sh_step[2];
    __shared__ int sh_code;
    const int nb = gridDim.x;
    // thread 0's scalars of the previous launch, loaded before the sums
    double rgamma_old = 0.0, pkp_old = 0.0, tol2 = 0.0;
    long long cg_max = 0;
    if (threadIdx.x == 0) {
        rgamma_old = st->rgamma[(k + 1) & 1];
        pkp_old = st->pkp[(k + 1) & 1];
        tol2 = st->tol2;
        cg_max = st->cg_max;
    }
    // this thread's first group of nodes, loaded before the sums so that the
    // loads overlap them (groups of G nodes with 16-byte accesses)
    constexpr int G = node_group(D, (int)sizeof(T)), E = G * D;
    const int64_t ng = nn / G, gstride = (int64_t)gridDim.x * kVT;
    int64_t gi = blockIdx.x * (int64_t)kVT + threadIdx.x;
    T zv[E], pv[E], sv[E], wv[E], xv[E], rv[E];
    if (gi < ng) {
        const int64_t i0 = gi * E;
        ld16(z + i0, zv);
        ld16(p + i0, pv);
        ld16(s + i0, sv);
        ld16(x + i0, xv);
        ld16(r + i0, rv);
    }
    fem::grid_dependency_wait();
    if (gi < ng) ld16(w + gi * E, wv);
    // r . r and r . z of the current residual (the previous kernel's block
    // partials, slot k & 1) and z . K z (the HVP's tile partials); loads in
    // batches of kB before the adds, so that they are in flight together
    constexpr int kB = 8;
    A acc[3] = {};
    const A* pin = partial + (size_t)(k & 1) * kVecBlocks * 2;
    for (int i = threadIdx.x; i < nb; i += kVT) {
        acc_add(acc[0], ld_acc(pin + 2 * i));
        acc_add(acc[1], ld_acc(pin + 2 * i + 1));
    }
    for (int t0 = threadIdx.x; t0 < n_tiles; t0 += kB * kVT) {
        A q[kB];
#pragma unroll
        for (int j = 0; j < kB; ++j) q[j] = t0 + j * kVT < n_tiles ? tile_partial<T>(tile_red, t0 + j * kVT) : A{};
#pragma unroll
        for (int j = 0; j < kB; ++j) acc_add(acc[2], q[j]);
    }
    block_sum<3>(acc, sh);
    // the scalar recurrences run in thread 0 alone and reach the block as
    // steps in the CG type.  With pkp = p^T K p and rgamma = 1 / gamma kept
    // from the previous launch: beta = gamma rgamma_old, beta gamma /
    // alpha_old = beta^2 pkp_old, so the only division on this path is
    // alpha = gamma / p^T K p (in the CG type; FP64 issues slowly here).
    double rr = 0.0, gamma = 0.0, pKp = 0.0;
    if (threadIdx.x == 0) {
        rr = widen(acc[0]);
        gamma = widen(acc[1]);
        const double delta = widen(acc[2]);
        int code = 0;
        double beta = 0.0;
        T alpha = T(0);
        if (rr <= tol2) {
            code = 1;
        } else if (k >= cg_max) {
            code = 3;
        } else {
            beta = k == 0 ? 0.0 : gamma * rgamma_old;
            pKp = k == 0 ? delta : delta - beta * beta * pkp_old;
            if (pKp > 0.0)
                alpha = (T)gamma / (T)pKp;
            else
                code = 2;  // non-positive curvature
        }
        sh_code = code;
        sh_step[0] = alpha;
        sh_step[1] = (T)beta;
    }
    __syncthreads();
    const int code = sh_code;
    if (code) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->rr = rr;
            st->k = code == 2 ? (int)k + 1 : (int)k;  // HVPs spent (the curvature test used this one)
            st->done = code;
        }
        return;
    }
    const T a = sh_step[0], bt = sh_step[1];
    A v[2] = {};
    while (gi < ng) {
        const int64_t i0 = gi * E;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            pv[e] = zv[e] + bt * pv[e];
            sv[e] = wv[e] + bt * sv[e];
            xv[e] += a * pv[e];
            rv[e] -= a * sv[e];
        }
        st16(p + i0, pv);
        st16(s + i0, sv);
        st16(x + i0, xv);
        st16(r + i0, rv);
        T Mv[E * D];
        ld16(Minv + gi * E * D, Mv);
#pragma unroll
        for (int q = 0; q < G; ++q)
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T t = Mv[(q * D + i) * D] * rv[q * D];
#pragma unroll
                for (int j = 1; j < D; ++j) t += Mv[(q * D + i) * D + j] * rv[q * D + j];
                zv[q * D + i] = t;
            }
        st16(z + i0, zv);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            acc_prod(v[0], rv[e], rv[e]);
            acc_prod(v[1], rv[e], zv[e]);
        }
        gi += gstride;
        if (gi < ng) {  // the next group
            const int64_t i1 = gi * E;
            ld16(z + i1, zv);
            ld16(p + i1, pv);
            ld16(s + i1, sv);
            ld16(w + i1, wv);
            ld16(x + i1, xv);
            ld16(r + i1, rv);
        }
    }
    for (int64_t n = ng * G + blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
        T rv[3] = {0, 0, 0}, zz[3];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int64_t i = n * D + c;
            const T pn = z[i] + bt * p[i];
            const T sn = w[i] + bt * s[i];
            p[i] = pn;
            s[i] = sn;
            x[i] += a * pn;
            rv[c] = r[i] - a * sn;
            r[i] = rv[c];
        }
        apply_block<D, T>(Minv, n, rv, zz);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            z[n * D + c] = zz[c];
            acc_prod(v[0], rv[c], rv[c]);
            acc_prod(v[1], rv[c], zz[c]);
        }
    }
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        A* pout = partial + (size_t)((k + 1) & 1) * kVecBlocks * 2;
        pout[2 * blockIdx.x] = v[0];
        pout[2 * blockIdx.x + 1] = v[1];
        if (blockIdx.x == 0) {  // read by launch k + 1
            st->rgamma[k & 1] = 1.0 / gamma;
            st->pkp[k & 1] = pKp;
        }
    }
}

// FP64 dot product a . b with a fixed summation order
template <typename TA, typename TB>
__global__ void __launch_bounds__(kVT) dot_kernel(int64_t n, const TA* a, const TB* b, DotState* ds,
                                                  double* partial) {
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT)
        v[0] = fma((double)a[i], (double)b[i], v[0]);
    double tot[1];
    if (grid_total<1>(v, tot, partial, &ds->counter) && threadIdx.x == 0) ds->value = tot[0];
}

// ---------------------------------------------------------------------------
// element-wise vector kernels
// ---------------------------------------------------------------------------
// du = (s1 - s0) ubar on prescribed DOFs, 0 elsewhere (FP64 and, if asked, FP32)
template <int D>
__global__ void predictor_increment(int64_t nn, const uint8_t* mask, const double* ubar, double ds,
                                    double* du, float* du32) {
    for (int64_t n = blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
        const uint8_t m = mask[n];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double v = ((m >> c) & 1) ? ds * ubar[n * D + c] : 0.0;
            du[n * D + c] = v;
            if (du32) du32[n * D + c] = (float)v;
        }
    }
}

__global__ void to_f32(int64_t n, const double* a, float* b) {
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT)
        b[i] = (float)a[i];
}

template <typename TS, typename TD>
__global__ void negate(int64_t n, const TS* a, TD* b) {
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT)
        b[i] = -(TD)a[i];
}

// dst = src with prescribed components zeroed (FP64 -> the CG dtype)
template <int D, typename TD>
__global__ void masked_copy(int64_t nn, const uint8_t* mask, const double* src, TD* dst) {
    for (int64_t n = blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
        const uint8_t m = mask[n];
#pragma unroll
        for (int c = 0; c < D; ++c) dst[n * D + c] = ((m >> c) & 1) ? TD(0) : (TD)src[n * D + c];
    }
}

template <typename TS>
__global__ void widen(int64_t n, const TS* a, double* b) {
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT)
        b[i] = (double)a[i];
}

// u += du on prescribed DOFs, u += x elsewhere
template <int D, typename T>
__global__ void apply_predictor(int64_t nn, const uint8_t* mask, double* u, const double* du, const T* x) {
    for (int64_t n = blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
        const uint8_t m = mask[n];
#pragma unroll
        for (int c = 0; c < D; ++c) u[n * D + c] += ((m >> c) & 1) ? du[n * D + c] : (double)x[n * D + c];
    }
}

template <int D>
__global__ void set_prescribed(int64_t nn, const uint8_t* mask, double* u, const double* ubar, double s) {
    for (int64_t n = blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
        const uint8_t m = mask[n];
#pragma unroll
        for (int c = 0; c < D; ++c)
            if ((m >> c) & 1) u[n * D + c] = s * ubar[n * D + c];
    }
}

// ut = u + alpha x
template <typename T>
__global__ void trial_point(int64_t n, const double* u, double alpha, const T* x, double* ut) {
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT)
        ut[i] = u[i] + alpha * (double)x[i];
}

// Minv_n = D_n^-1 through the Cholesky factor D_n = L L^T (FP64 per node):
// L^-1 by forward substitution, Minv = L^-T L^-1.  A non-positive pivot sets
// *bad and leaves the identity.
// uc = u on prescribed components, 0 on free ones
template <int D>
__global__ void prescribed_part(int64_t nn, const uint8_t* mask, const double* u, double* uc) {
    for (int64_t n = blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
        const uint8_t m = mask[n];
#pragma unroll
        for (int c = 0; c < D; ++c) uc[n * D + c] = ((m >> c) & 1) ? u[n * D + c] : 0.0;
    }
}

// a = uc - lam (the adjoint weights: u_c on prescribed DOFs, -lam on free
// ones, where lam vanishes on prescribed DOFs), FP64 and optionally FP32
__global__ void adjoint_weights(int64_t n, const double* uc, const double* lam, double* a, float* a32) {
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT) {
        const double x = uc[i] - lam[i];
        a[i] = x;
        if (a32) a32[i] = (float)x;
    }
}

// res = rhs - res (res holds M K M lam on entry)
__global__ void residual_update(int64_t n, const double* rhs, double* res) {
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT)
        res[i] = rhs[i] - res[i];
}

// y += x
__global__ void add_into(int64_t n, const double* x, double* y) {
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT) y[i] += x[i];
}

// g = g_mu + ratio g_lam per element (lambda_e = ratio mu_e)
__global__ void tied_moduli(int64_t n, double* g, const double* glam, double ratio) {
    for (int64_t i = blockIdx.x * (int64_t)kVT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVT)
        g[i] = fma(ratio, glam[i], g[i]);
}

template <int D, typename T>
__global__ void block_jacobi_inverse(int64_t nn, const T* Db, T* Minv, int* bad) {
    if constexpr (sizeof(T) == 4) {
        // FP32 CG: the closed-form inverse adj(A) / det A in FP32, with the
        // block called SPD when its leading principal minors are positive
        // (Sylvester's criterion); the nodal blocks are symmetric and well
        // conditioned, so FP32 rounding changes the preconditioner, not the
        // converged solution
        for (int64_t n = blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
            float A[D][D], Mi[D][D];
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) A[i][j] = (float)Db[n * D * D + i * D + j];
            float det, m2;
            if constexpr (D == 3) {
                const float c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
                const float c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
                const float c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
                m2 = A[0][0] * A[1][1] - A[0][1] * A[1][0];
                det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
                const float rd = 1.0f / det;
                Mi[0][0] = c00 * rd;
                Mi[1][0] = c01 * rd;
                Mi[2][0] = c02 * rd;
                Mi[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * rd;
                Mi[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * rd;
                Mi[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * rd;
                Mi[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * rd;
                Mi[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * rd;
                Mi[2][2] = m2 * rd;
            } else {
                m2 = A[0][0];
                det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
                const float rd = 1.0f / det;
                Mi[0][0] = A[1][1] * rd;
                Mi[0][1] = -A[0][1] * rd;
                Mi[1][0] = -A[1][0] * rd;
                Mi[1][1] = A[0][0] * rd;
            }
            const bool ok = A[0][0] > 0.f && m2 > 0.f && det > 0.f && isfinite(det);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) Minv[n * D * D + i * D + j] = ok ? Mi[i][j] : (i == j ? 1.f : 0.f);
            if (!ok) atomicOr(bad, 1);
        }
    } else {
    for (int64_t n = blockIdx.x * (int64_t)kVT + threadIdx.x; n < nn; n += (int64_t)gridDim.x * kVT) {
        double A[D][D], L[D][D] = {}, Li[D][D] = {};
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) A[i][j] = (double)Db[n * D * D + i * D + j];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                double s = A[i][j];
#pragma unroll
                for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
                if (i == j) {
                    if (!(s > 0.0)) {
                        ok = false;
                        s = 1.0;
                    }
                    L[i][i] = sqrt(s);
                } else {
                    L[i][j] = s / L[j][j];
                }
            }
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
            for (int i = 0; i < D; ++i) {
                double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < i; ++k) s -= L[i][k] * Li[k][j];
                Li[i][j] = s / L[i][i];
            }
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) s += Li[k][i] * Li[k][j];
                Minv[n * D * D + i * D + j] = ok ? (T)s : (T)(i == j ? 1.0 : 0.0);
            }
        if (!ok) atomicOr(bad, 1);
    }
    }
}

int grid_for(int64_t work) {
    const int64_t g = (work + kVT - 1) / kVT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, kVecBlocks));
}

fem_status fail(fem_status s, const std::string& msg) { return femi::set_error(s, msg); }

#define CUDA_TRY(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(FEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define FEM_TRY(call)                      \
    do {                                   \
        fem_status s_ = (call);            \
        if (s_ != FEM_OK) return s_;       \
    } while (0)

}  // namespace

namespace femi {

struct SolverWork {
    int64_t nn = 0, nd = 0;
    int D = 0;
    std::vector<void*> allocs;
    // FP64 vectors
    double *r = nullptr, *t = nullptr, *du = nullptr, *ut = nullptr;
    std::vector<double*> saves;  // one per bisection depth
    float *u32 = nullptr, *du32 = nullptr;
    // CG vectors, index 0: FP64, 1: FP32 (allocated on first use)
    void *b[2] = {}, *x[2] = {}, *res[2] = {}, *z[2] = {}, *p[2] = {}, *q[2] = {}, *s[2] = {}, *Minv[2] = {},
         *Db[2] = {};
    double* partial = nullptr;
    CgState* cg = nullptr;
    DotState* dot = nullptr;
    double* scal = nullptr;  // energy output (4 doubles)
    double* glam = nullptr;  // compliance gradient: per-element g_lam (allocated on first use)
    double* adj = nullptr;   // compliance gradient: correction of the refined adjoint solve
    int* bad = nullptr;
    // pinned host mirror
    struct Host {
        CgState cg;
        DotState dot;
        double scal[4];
        int done[2];
        int bad;
        int status;
    }* h = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

void solver_free(fem_mesh* m) {
    SolverWork* w = m ? m->solver : nullptr;
    if (!w) return;
    for (void* p : w->allocs) cudaFree(p);
    for (double* p : w->saves) cudaFree(p);
    if (w->h) cudaFreeHost(w->h);
    for (auto& e : w->ev)
        if (e) cudaEventDestroy(e);
    delete w;
    m->solver = nullptr;
}

}  // namespace femi

namespace {

using femi::SolverWork;

template <typename T>
fem_status dalloc(SolverWork* w, T** p, size_t n) {
    void* q = nullptr;
    CUDA_TRY(cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)));
    w->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return FEM_OK;
}

fem_status ensure_work(fem_mesh* m, int cg_dtype) {
    if (!m->solver) {
        auto* w = new SolverWork();
        m->solver = w;
        w->nn = m->info.n_nodes;
        w->D = m->dim;
        w->nd = w->nn * w->D;
        FEM_TRY(dalloc(w, &w->r, w->nd));
        FEM_TRY(dalloc(w, &w->t, w->nd));
        FEM_TRY(dalloc(w, &w->du, w->nd));
        FEM_TRY(dalloc(w, &w->ut, w->nd));
        // dot_kernel: kMaxRedBlocks slots; PCG: 2 x kVecBlocks x 2 (8-byte) slots
        FEM_TRY(dalloc(w, &w->partial, (size_t)std::max(kMaxRedBlocks, 2 * kVecBlocks) * 2));
        FEM_TRY(dalloc(w, &w->cg, 1));
        FEM_TRY(dalloc(w, &w->dot, 1));
        FEM_TRY(dalloc(w, &w->scal, 4));
        FEM_TRY(dalloc(w, &w->bad, 1));
        CUDA_TRY(cudaMemset(w->cg, 0, sizeof(CgState)));
        CUDA_TRY(cudaMemset(w->dot, 0, sizeof(DotState)));
        void* h = nullptr;
        CUDA_TRY(cudaMallocHost(&h, sizeof(SolverWork::Host)));
        w->h = static_cast<SolverWork::Host*>(h);
        std::memset(w->h, 0, sizeof(SolverWork::Host));
        for (auto& e : w->ev) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    SolverWork* w = m->solver;
    const int pi = cg_dtype == FEM_F64 ? 0 : 1;
    if (!w->b[pi]) {
        const size_t ts = pi == 0 ? 8 : 4;
        void** vecs[] = {&w->b[pi], &w->x[pi], &w->res[pi], &w->z[pi], &w->p[pi], &w->q[pi], &w->s[pi]};
        for (void** v : vecs) {
            uint8_t* q = nullptr;
            FEM_TRY(dalloc(w, &q, (size_t)w->nd * ts));
            *v = q;
        }
        uint8_t* q = nullptr;
        FEM_TRY(dalloc(w, &q, (size_t)w->nn * w->D * w->D * ts));
        w->Minv[pi] = q;
        FEM_TRY(dalloc(w, &q, (size_t)w->nn * w->D * w->D * ts));
        w->Db[pi] = q;
        if (pi == 1) {
            FEM_TRY(dalloc(w, &w->u32, w->nd));
            FEM_TRY(dalloc(w, &w->du32, w->nd));
        }
    }
    return FEM_OK;
}

// One load increment and its bisection; mirrors the oracle step for step.
class Stepper {
public:
    Stepper(fem_mesh* m, const fem_newton_opts& o, fem_newton_stats* stats, cudaStream_t st)
        : m_(m), o_(o), stats_(stats), st_(st), w_(m->solver), D_(m->dim) {
        dt_ = o.cg_dtype;
        pi_ = dt_ == FEM_F64 ? 0 : 1;
        cg_max_ = o.cg_max > 0 ? o.cg_max : 10 * w_->nd;
    }

    // returns 0 on success or the oracle's failure code (3 inverted, 5 not
    // SPD, 6 not converged, 7 line search); a CUDA failure sets *err
    int step_rec(double* u, const double* ubar, double s0, double s1, int depth, fem_status* err) {
        if ((int)w_->saves.size() <= depth) {
            double* sv = nullptr;
            if (cudaMalloc(&sv, sizeof(double) * w_->nd) != cudaSuccess) {
                *err = fail(FEM_ERR_CUDA, "cudaMalloc of a bisection save vector failed");
                return -1;
            }
            w_->saves.push_back(sv);
        }
        double* save = w_->saves[depth];
        if (cudaMemcpyAsync(save, u, sizeof(double) * w_->nd, cudaMemcpyDeviceToDevice, st_) != cudaSuccess) {
            *err = fail(FEM_ERR_CUDA, "cudaMemcpyAsync (save) failed");
            return -1;
        }
        int rc = increment(u, ubar, s0, s1, err);
        if (*err != FEM_OK) return -1;
        if (rc != 0 && depth < o_.max_bisect) {
            if (cudaMemcpyAsync(u, save, sizeof(double) * w_->nd, cudaMemcpyDeviceToDevice, st_) != cudaSuccess) {
                *err = fail(FEM_ERR_CUDA, "cudaMemcpyAsync (restore) failed");
                return -1;
            }
            stats_->bisections++;
            const double sm = 0.5 * (s0 + s1);
            rc = step_rec(u, ubar, s0, sm, depth + 1, err);
            if (rc == 0 && *err == FEM_OK) rc = step_rec(u, ubar, sm, s1, depth + 1, err);
        }
        return rc;
    }

    // x = PCG solution of M K(u) M x = M b from 0 to ||res|| <= rtol ||M b||
    // (b, x FP64); returns 0, 2 (non-positive curvature) or 3 (iteration cap)
    int tangent_solve(const double* u, const double* b, double* x, double rtol, int64_t* iters, fem_status* err) {
        const void* ucg = cg_state(u);
        const int rc = build_block_jacobi(ucg, err);
        if (*err != FEM_OK) return -1;
        if (rc != 0) return 5;
        const int gn = grid_nodes(), gd = grid_dofs();
        if (D_ == 2) {
            if (pi_ == 0)
                masked_copy<2, double><<<gn, kVT, 0, st_>>>(w_->nn, m_->node_mask, b, (double*)w_->b[0]);
            else
                masked_copy<2, float><<<gn, kVT, 0, st_>>>(w_->nn, m_->node_mask, b, (float*)w_->b[1]);
        } else {
            if (pi_ == 0)
                masked_copy<3, double><<<gn, kVT, 0, st_>>>(w_->nn, m_->node_mask, b, (double*)w_->b[0]);
            else
                masked_copy<3, float><<<gn, kVT, 0, st_>>>(w_->nn, m_->node_mask, b, (float*)w_->b[1]);
        }
        double bb = 0.0;
        *err = dot(w_->b[pi_], dt_, w_->b[pi_], dt_, &bb);
        if (*err != FEM_OK) return -1;
        *err = pcg(ucg, rtol * std::sqrt(bb), iters);
        if (*err != FEM_OK) return -1;
        if (pi_ == 0)
            widen<double><<<gd, kVT, 0, st_>>>(w_->nd, (const double*)w_->x[0], x);
        else
            widen<float><<<gd, kVT, 0, st_>>>(w_->nd, (const float*)w_->x[1], x);
        if (cudaStreamSynchronize(st_) != cudaSuccess) {
            *err = fail(FEM_ERR_CUDA, "cudaStreamSynchronize failed");
            return -1;
        }
        const int done = w_->h->cg.done;
        return done == 1 ? 0 : done;
    }

private:
    fem_mesh* m_;
    fem_newton_opts o_;
    fem_newton_stats* stats_;
    cudaStream_t st_;
    SolverWork* w_;
    int D_, dt_, pi_;
    int64_t cg_max_;
    bool lin_ = false;  // the PCG's HVPs read a stored linearisation

    int grid_nodes() const { return grid_for(w_->nn); }
    int grid_dofs() const { return grid_for(w_->nd); }

    fem_status sync() {
        CUDA_TRY(cudaStreamSynchronize(st_));
        return FEM_OK;
    }

    // FP64 dot a . b (ta, tb: FEM_F64 / FEM_F32), returned to the host
    fem_status dot(const void* a, int ta, const void* b, int tb, double* out) {
        const int g = grid_dofs();
        const int64_t n = w_->nd;
        if (ta == FEM_F64 && tb == FEM_F64)
            dot_kernel<double, double><<<g, kVT, 0, st_>>>(n, (const double*)a, (const double*)b, w_->dot, w_->partial);
        else if (ta == FEM_F64)
            dot_kernel<double, float><<<g, kVT, 0, st_>>>(n, (const double*)a, (const float*)b, w_->dot, w_->partial);
        else if (tb == FEM_F64)
            dot_kernel<float, double><<<g, kVT, 0, st_>>>(n, (const float*)a, (const double*)b, w_->dot, w_->partial);
        else
            dot_kernel<float, float><<<g, kVT, 0, st_>>>(n, (const float*)a, (const float*)b, w_->dot, w_->partial);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(&w_->h->dot, w_->dot, sizeof(DotState), cudaMemcpyDeviceToHost, st_));
        FEM_TRY(sync());
        *out = w_->h->dot.value;
        return FEM_OK;
    }

    // Psi(u) and the roundoff scale S (FP64).  With a neural constitutive
    // model the call also leaves the network's gradient coefficients at u, so
    // that residual(u, r, true) right after it skips the network (bitwise the
    // same result: the same coefficients at the same state).
    fem_status energy(const double* u, double* psi, double* S) {
        FEM_TRY(femi::run_op(m_, FEM_F64, fem::OP_ENERGY, u, nullptr, nullptr, w_->scal,
                             m_->ncm ? femi::kFlagNcmGrad : 0u, st_, nullptr));
        CUDA_TRY(cudaMemcpyAsync(w_->h->scal, w_->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, st_));
        FEM_TRY(sync());
        *psi = w_->h->scal[0];
        *S = w_->h->scal[1];
        return FEM_OK;
    }

    // same_as_energy: u is the state of the last energy call, and no other
    // FP64 call of the network has run since
    fem_status residual(const double* u, double* r, bool same_as_energy = false) {
        const unsigned keep = (same_as_energy && m_->ncm) ? femi::kFlagNcmCurrent : 0u;
        return femi::run_op(m_, FEM_F64, fem::OP_RESIDUAL, u, nullptr, r, nullptr, FEM_MASK_OUT | keep, st_, nullptr);
    }

    // the state the CG's element kernels see: u itself (FP64) or its FP32 shadow
    const void* cg_state(const double* u) {
        if (pi_ == 0) return u;
        to_f32<<<grid_dofs(), kVT, 0, st_>>>(w_->nd, u, w_->u32);
        return w_->u32;
    }

    // block-Jacobi (or learned) preconditioner at u; returns 5 when a block
    // is not SPD
    int build_block_jacobi(const void* ucg, fem_status* err) {
        if (o_.precond == FEM_PC_LEARNED) {
            *err = femi::lp_precondition(o_.learned, m_, static_cast<const float*>(ucg),
                                         static_cast<float*>(w_->Minv[1]), st_);
            return *err == FEM_OK ? 0 : -1;
        }
        *err = femi::run_op(m_, dt_, fem::OP_BLOCKDIAG, ucg, nullptr, w_->Db[pi_], nullptr, 0, st_, nullptr);
        if (*err != FEM_OK) return -1;
        if (cudaMemsetAsync(w_->bad, 0, sizeof(int), st_) != cudaSuccess) {
            *err = fail(FEM_ERR_CUDA, "cudaMemsetAsync failed");
            return -1;
        }
        const int g = grid_nodes();
        if (D_ == 2) {
            if (pi_ == 0)
                block_jacobi_inverse<2, double><<<g, kVT, 0, st_>>>(w_->nn, (const double*)w_->Db[0], (double*)w_->Minv[0], w_->bad);
            else
                block_jacobi_inverse<2, float><<<g, kVT, 0, st_>>>(w_->nn, (const float*)w_->Db[1], (float*)w_->Minv[1], w_->bad);
        } else {
            if (pi_ == 0)
                block_jacobi_inverse<3, double><<<g, kVT, 0, st_>>>(w_->nn, (const double*)w_->Db[0], (double*)w_->Minv[0], w_->bad);
            else
                block_jacobi_inverse<3, float><<<g, kVT, 0, st_>>>(w_->nn, (const float*)w_->Db[1], (float*)w_->Minv[1], w_->bad);
        }
        if (cudaMemcpyAsync(&w_->h->bad, w_->bad, sizeof(int), cudaMemcpyDeviceToHost, st_) != cudaSuccess ||
            cudaStreamSynchronize(st_) != cudaSuccess) {
            *err = fail(FEM_ERR_CUDA, "block-Jacobi readback failed");
            return -1;
        }
        return w_->h->bad ? 5 : 0;
    }

    // grid of cg_init and cg_step (one group of node_group nodes per thread)
    template <int D, typename T>
    int cg_grid() const {
        return grid_for(w_->nn / node_group(D, (int)sizeof(T)) + 1);
    }

    template <int D, typename T>
    fem_status launch_cg_iteration(const void* ucg, long long k) {
        SolverWork* w = w_;
        const int pi = pi_;
        using A = typename AccT<T>::type;
        // w = K z with z . K z (fused), then the update
        // (both as programmatic dependent launches: each kernel's blocks are
        // placed while the previous kernel drains)
        // the state is fixed: a neural constitutive model's coefficients at
        // ucg are current (the preconditioner build evaluated them), and a
        // Neo-Hookean HVP reads the linearisation stored by pcg_t
        const unsigned fixed_state = m_->ncm ? femi::kFlagNcmCurrent : (lin_ ? femi::kFlagUseLin : 0u);
        FEM_TRY(femi::run_op(m_, dt_, fem::OP_HVP, ucg, w->z[pi], w->q[pi], nullptr,
                             FEM_MASK_IN | FEM_MASK_OUT | fixed_state, st_, &w->cg->done, /*vkv_tiles=*/1));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)cg_grid<D, T>());
        cfg.blockDim = dim3(kVT);
        cfg.stream = st_;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CUDA_TRY(cudaLaunchKernelEx(&cfg, cg_step<D, T>, (int64_t)w->nn, k, (T*)w->x[pi], (T*)w->res[pi],
                                    (T*)w->z[pi], (T*)w->p[pi], (T*)w->s[pi], (const T*)w->q[pi],
                                    (const T*)w->Minv[pi], w->cg, reinterpret_cast<A*>(w->partial),
                                    femi::tile_partials(m_), m_->info.n_tiles));
        return FEM_OK;
    }

    // PCG on M K M x = b (b in w->b) from x = 0 to ||res|| <= tol; the
    // number of HVPs goes to *iters
    template <int D, typename T>
    fem_status pcg_t(const void* ucg, double tol, int64_t* iters) {
        SolverWork* w = w_;
        const int pi = pi_;
        SolverWork::Host* h = w->h;
        h->cg.tol2 = tol * tol;
        h->cg.cg_max = cg_max_;
        // tol2 and cg_max are set per solve; cg_init resets done and k, and the
        // rest is written by each launch before the next one reads it
        CUDA_TRY(cudaMemcpyAsync(&w->cg->tol2, &h->cg.tol2, sizeof(double), cudaMemcpyHostToDevice, st_));
        CUDA_TRY(cudaMemcpyAsync(&w->cg->cg_max, &h->cg.cg_max, sizeof(long long), cudaMemcpyHostToDevice, st_));
        using A = typename AccT<T>::type;
        // the linearisation at ucg, read by every HVP of the solve
        lin_ = !m_->ncm;
        if (lin_)
            FEM_TRY(femi::run_op(m_, dt_, fem::OP_LINEARIZE, ucg, nullptr, nullptr, nullptr, 0, st_, nullptr));
        cg_init<D, T><<<cg_grid<D, T>(), kVT, 0, st_>>>(w->nn, (const T*)w->b[pi], (T*)w->x[pi], (T*)w->res[pi],
                                                        (T*)w->z[pi], (T*)w->p[pi], (T*)w->s[pi],
                                                        (const T*)w->Minv[pi], w->cg, reinterpret_cast<A*>(w->partial));
        CUDA_TRY(cudaGetLastError());
        const int B = o_.cg_batch > 0 ? o_.cg_batch : 8;
        // the stop is seen one launch after the update that reaches it: the
        // launches run past cg_max so that the cap is always taken
        const int64_t max_batches = cg_max_ / B + 3;
        for (int64_t j = 0; j < max_batches; ++j) {
            for (int i = 0; i < B; ++i) FEM_TRY((launch_cg_iteration<D, T>(ucg, (long long)(j * B + i))));
            CUDA_TRY(cudaMemcpyAsync(&h->done[j & 1], &w->cg->done, sizeof(int), cudaMemcpyDeviceToHost, st_));
            CUDA_TRY(cudaEventRecord(w->ev[j & 1], st_));
            if (j >= 1) {
                CUDA_TRY(cudaEventSynchronize(w->ev[(j - 1) & 1]));
                if (h->done[(j - 1) & 1]) break;
            }
        }
        CUDA_TRY(cudaMemcpyAsync(&h->cg, w->cg, sizeof(CgState), cudaMemcpyDeviceToHost, st_));
        FEM_TRY(sync());
        if (!h->cg.done) return fail(FEM_ERR_CUDA, "PCG ended without a final state");
        if (h->cg.done == 2 && h->cg.k == 1)  // curvature test failed at once: take d = M b
            CUDA_TRY(cudaMemcpyAsync(w->x[pi], w->z[pi], (size_t)w->nd * sizeof(T), cudaMemcpyDeviceToDevice, st_));
        *iters = h->cg.k;
        return FEM_OK;
    }

    fem_status pcg(const void* ucg, double tol, int64_t* iters) {
        if (D_ == 2) return pi_ == 0 ? pcg_t<2, double>(ucg, tol, iters) : pcg_t<2, float>(ucg, tol, iters);
        return pi_ == 0 ? pcg_t<3, double>(ucg, tol, iters) : pcg_t<3, float>(ucg, tol, iters);
    }

    // b = -src (src FP64 or the CG dtype)
    void set_rhs_neg(const void* src, int src_dt) {
        const int g = grid_dofs();
        if (pi_ == 0)
            negate<double, double><<<g, kVT, 0, st_>>>(w_->nd, (const double*)src, (double*)w_->b[0]);
        else if (src_dt == FEM_F64)
            negate<double, float><<<g, kVT, 0, st_>>>(w_->nd, (const double*)src, (float*)w_->b[1]);
        else
            negate<float, float><<<g, kVT, 0, st_>>>(w_->nd, (const float*)src, (float*)w_->b[1]);
    }

    int increment(double* u, const double* ubar, double s0, double s1, fem_status* err) {
#define STEP_TRY(call)             \
    do {                           \
        *err = (call);             \
        if (*err != FEM_OK) return -1; \
    } while (0)
        SolverWork* w = w_;
        const int64_t nn = w->nn, nd = w->nd;
        const int gn = grid_nodes(), gd = grid_dofs();
        // 1-2: prescribed increment and linearised predictor
        if (D_ == 2)
            predictor_increment<2><<<gn, kVT, 0, st_>>>(nn, m_->node_mask, ubar, s1 - s0, w->du, pi_ ? w->du32 : nullptr);
        else
            predictor_increment<3><<<gn, kVT, 0, st_>>>(nn, m_->node_mask, ubar, s1 - s0, w->du, pi_ ? w->du32 : nullptr);
        const void* ucg = cg_state(u);
        void* tv = pi_ == 0 ? (void*)w->t : w->q[1];  // predictor rhs in the CG dtype
        STEP_TRY(femi::run_op(m_, dt_, fem::OP_HVP, ucg, pi_ == 0 ? (const void*)w->du : (const void*)w->du32, tv,
                              nullptr, FEM_MASK_OUT, st_, nullptr));
        double r0sq = 0.0;
        STEP_TRY(dot(tv, dt_, tv, dt_, &r0sq));
        double r0 = std::sqrt(r0sq);
        if (!std::isfinite(r0)) return 3;
        if (r0 > 0.0) {
            const int rc = build_block_jacobi(ucg, err);
            if (rc != 0) return rc;
            set_rhs_neg(tv, dt_);
            int64_t it = 0;
            STEP_TRY(pcg(ucg, o_.predictor_rtol * r0, &it));
            stats_->cg_iters += it;
            if (D_ == 2) {
                if (pi_ == 0)
                    apply_predictor<2, double><<<gn, kVT, 0, st_>>>(nn, m_->node_mask, u, w->du, (const double*)w->x[0]);
                else
                    apply_predictor<2, float><<<gn, kVT, 0, st_>>>(nn, m_->node_mask, u, w->du, (const float*)w->x[1]);
            } else {
                if (pi_ == 0)
                    apply_predictor<3, double><<<gn, kVT, 0, st_>>>(nn, m_->node_mask, u, w->du, (const double*)w->x[0]);
                else
                    apply_predictor<3, float><<<gn, kVT, 0, st_>>>(nn, m_->node_mask, u, w->du, (const float*)w->x[1]);
            }
        }
        if (D_ == 2)
            set_prescribed<2><<<gn, kVT, 0, st_>>>(nn, m_->node_mask, u, ubar, s1);
        else
            set_prescribed<3><<<gn, kVT, 0, st_>>>(nn, m_->node_mask, u, ubar, s1);
        double psi = 0.0, S = 0.0;
        STEP_TRY(energy(u, &psi, &S));
        if (!std::isfinite(psi)) return 3;
        STEP_TRY(residual(u, w->r, true));
        double rsq = 0.0;
        STEP_TRY(dot(w->r, FEM_F64, w->r, FEM_F64, &rsq));
        double rn = std::sqrt(rsq);
        if (!(r0 > 0.0)) r0 = rn;
        stats_->r0_norm = r0;
        // 3: Newton loop
        for (int it = 0; it <= o_.newton_max; ++it) {
            stats_->r_norm = rn;
            if (rn <= o_.newton_rtol * r0) return 0;
            if (it == o_.newton_max) return 6;
            stats_->newton_iters++;
            const double eta = std::min(o_.eta_max, std::sqrt(rn / r0));
            ucg = cg_state(u);
            const int rc = build_block_jacobi(ucg, err);
            if (rc != 0) return rc;
            set_rhs_neg(w->r, FEM_F64);
            int64_t cgit = 0;
            STEP_TRY(pcg(ucg, eta * rn, &cgit));
            stats_->cg_iters += cgit;
            const void* xd = w->x[pi_];
            double g = 0.0;
            STEP_TRY(dot(w->r, FEM_F64, xd, dt_, &g));
            double alpha = 1.0;
            bool ok = false;
            for (int ls = 0; ls <= o_.ls_max; ++ls) {
                if (pi_ == 0)
                    trial_point<double><<<gd, kVT, 0, st_>>>(nd, u, alpha, (const double*)xd, w->ut);
                else
                    trial_point<float><<<gd, kVT, 0, st_>>>(nd, u, alpha, (const float*)xd, w->ut);
                double pt = 0.0, St = 0.0;
                STEP_TRY(energy(w->ut, &pt, &St));
                if (std::isfinite(pt)) {
                    if (pt <= psi + o_.armijo_c * alpha * g) {
                        ok = true;
                    } else if (std::fabs(pt - psi) <= 16.0 * kEps * S) {
                        STEP_TRY(residual(w->ut, w->t, true));
                        double rtsq = 0.0;
                        STEP_TRY(dot(w->t, FEM_F64, w->t, FEM_F64, &rtsq));
                        if (std::sqrt(rtsq) < rn) ok = true;
                    }
                }
                if (ok) {
                    psi = pt;
                    S = St;
                    break;
                }
                alpha *= 0.5;
                stats_->ls_halvings++;
            }
            if (!ok) return 7;
            if (cudaMemcpyAsync(u, w->ut, sizeof(double) * nd, cudaMemcpyDeviceToDevice, st_) != cudaSuccess) {
                *err = fail(FEM_ERR_CUDA, "cudaMemcpyAsync (accept) failed");
                return -1;
            }
            // u is the accepted trial state, the last one the energy saw
            STEP_TRY(residual(u, w->r, true));
            STEP_TRY(dot(w->r, FEM_F64, w->r, FEM_F64, &rsq));
            rn = std::sqrt(rsq);
        }
        return 6;
#undef STEP_TRY
    }

    static constexpr double kEps = 2.220446049250313e-16;
};

fem_status status_of(int rc) {
    switch (rc) {
        case 0: return FEM_OK;
        case 3: return FEM_ERR_INVERTED;
        case 5: return FEM_ERR_NOT_SPD;
        case 6: return FEM_ERR_NOT_CONVERGED;
        case 7: return FEM_ERR_LINESEARCH;
        default: return FEM_ERR_CUDA;
    }
}

}  // namespace

extern "C" {

fem_status fem_newton_default_opts(fem_newton_opts* o) {
    if (!o) return fail(FEM_ERR_ARG, "null options");
    std::memset(o, 0, sizeof *o);
    o->cg_dtype = FEM_F64;
    o->precond = FEM_PC_BLOCK_JACOBI;
    o->newton_rtol = 1e-8;
    o->newton_max = 50;
    o->eta_max = 0.1;
    o->cg_max = 0;
    o->predictor_rtol = 1e-2;
    o->armijo_c = 1e-4;
    o->ls_max = 20;
    o->max_bisect = 5;
    o->cg_batch = 8;
    o->learned = nullptr;
    return FEM_OK;
}

fem_status fem_newton_step(fem_mesh* m, double* u, const double* ubar, double s_prev, double s,
                           const fem_newton_opts* opts, fem_newton_stats* stats, void* stream) {
    if (!m || !u || !ubar || !stats) return fail(FEM_ERR_ARG, "null mesh, u, ubar or stats");
    fem_newton_opts o;
    if (opts)
        o = *opts;
    else
        fem_newton_default_opts(&o);
    if (o.cg_dtype != FEM_F64 && o.cg_dtype != FEM_F32) return fail(FEM_ERR_ARG, "cg_dtype must be FEM_F64 or FEM_F32");
    if (o.cg_dtype == FEM_F32 && m->precision != FEM_PREC_MIXED)
        return fail(FEM_ERR_ARG, "cg_dtype FEM_F32 needs a mesh created with FEM_PREC_MIXED");
    if (o.precond != FEM_PC_BLOCK_JACOBI && o.precond != FEM_PC_LEARNED) return fail(FEM_ERR_ARG, "unknown preconditioner");
    if (o.precond == FEM_PC_LEARNED && (o.cg_dtype != FEM_F32 || m->dim != 3 || !o.learned))
        return fail(FEM_ERR_ARG, "FEM_PC_LEARNED needs cg_dtype FEM_F32, a 3D mesh and a fem_lp handle");
    if (o.newton_max < 0 || o.ls_max < 0 || o.max_bisect < 0 || o.cg_max < 0)
        return fail(FEM_ERR_ARG, "negative iteration limit");
    if (!(s >= s_prev) || !std::isfinite(s) || !std::isfinite(s_prev)) return fail(FEM_ERR_ARG, "need finite s >= s_prev");
    std::memset(stats, 0, sizeof *stats);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FEM_TRY(ensure_work(m, o.cg_dtype));
    SolverWork* w = m->solver;
    // keep the caller's status word: trial states of the line search may
    // raise the inverted flag, which the step handles itself
    CUDA_TRY(cudaMemcpyAsync(&w->h->status, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    const int status_in = w->h->status;
    Stepper stepper(m, o, stats, st);
    fem_status err = FEM_OK;
    const int rc = stepper.step_rec(u, ubar, s_prev, s, 0, &err);
    w->h->status = status_in;
    CUDA_TRY(cudaMemcpyAsync(m->status, &w->h->status, sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (err != FEM_OK) {
        stats->status = err;
        return err;
    }
    const fem_status fs = status_of(rc);
    stats->status = fs;
    if (rc != 0)
        return fail(fs, "fem_newton_step: " + std::string(rc == 3   ? "inverted elements"
                                                                   : rc == 5 ? "a nodal block is not SPD"
                                                                   : rc == 6 ? "Newton iteration cap reached"
                                                                             : "line search failed") +
                                       " after all bisections");
    return FEM_OK;
}

fem_status fem_tangent_solve(fem_mesh* m, int cg_dtype, const double* u, const double* b, double* x,
                             double rtol, int64_t cg_max, int64_t* iters, void* stream) {
    if (!m || !u || !b || !x) return fail(FEM_ERR_ARG, "null mesh, u, b or x");
    if (cg_dtype != FEM_F64 && cg_dtype != FEM_F32) return fail(FEM_ERR_ARG, "cg_dtype must be FEM_F64 or FEM_F32");
    if (cg_dtype == FEM_F32 && m->precision != FEM_PREC_MIXED)
        return fail(FEM_ERR_ARG, "cg_dtype FEM_F32 needs a mesh created with FEM_PREC_MIXED");
    if (!(rtol > 0.0) || cg_max < 0) return fail(FEM_ERR_ARG, "need rtol > 0 and cg_max >= 0");
    fem_newton_opts o;
    fem_newton_default_opts(&o);
    o.cg_dtype = cg_dtype;
    o.cg_max = cg_max;
    fem_newton_stats stats{};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FEM_TRY(ensure_work(m, cg_dtype));
    Stepper stepper(m, o, &stats, st);
    fem_status err = FEM_OK;
    int64_t it = 0;
    const int rc = stepper.tangent_solve(u, b, x, rtol, &it, &err);
    if (iters) *iters = it;
    if (err != FEM_OK) return err;
    if (rc == 5) return fail(FEM_ERR_NOT_SPD, "fem_tangent_solve: a nodal diagonal block is not SPD");
    if (rc == 2) return fail(FEM_ERR_NEG_CURVATURE, "fem_tangent_solve: p^T K p <= 0 (K is not positive definite)");
    if (rc == 3) return fail(FEM_ERR_NOT_CONVERGED, "fem_tangent_solve: iteration cap reached");
    return FEM_OK;
}

fem_status fem_compliance_gradient(fem_mesh* m, const double* u, double ratio, double rtol, int cg_dtype,
                                   int vjp_dtype, double* dmu, double* c_dev, int64_t* iters, void* stream) {
    if (!m || !u || !dmu || !c_dev) return fail(FEM_ERR_ARG, "null mesh, u, dmu or c");
    if (cg_dtype != FEM_F64 && cg_dtype != FEM_F32) return fail(FEM_ERR_ARG, "cg_dtype must be FEM_F64 or FEM_F32");
    if (vjp_dtype != FEM_F64 && vjp_dtype != FEM_F32) return fail(FEM_ERR_ARG, "vjp_dtype must be FEM_F64 or FEM_F32");
    if ((cg_dtype == FEM_F32 || vjp_dtype == FEM_F32) && m->precision != FEM_PREC_MIXED)
        return fail(FEM_ERR_ARG, "FEM_F32 needs a mesh created with FEM_PREC_MIXED");
    if (!(rtol > 0.0) || !std::isfinite(ratio)) return fail(FEM_ERR_ARG, "need rtol > 0 and a finite ratio");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FEM_TRY(ensure_work(m, cg_dtype));
    if (vjp_dtype == FEM_F32) FEM_TRY(ensure_work(m, FEM_F32));
    SolverWork* w = m->solver;
    if (!w->glam) FEM_TRY(dalloc(w, &w->glam, (size_t)m->info.n_elems));
    const int gn = grid_for(w->nn), gd = grid_for(w->nd);
    double* uc = w->du;   // prescribed part of u
    double* r = w->r;     // unmasked residual at u
    double* rhs = w->t;   // K_fc u_c (free rows)
    double* lam = w->ut;  // adjoint solution
    // 1. c = u_c^T r(u): the work of the prescribed displacements
    if (m->dim == 2)
        prescribed_part<2><<<gn, kVT, 0, st>>>(w->nn, m->node_mask, u, uc);
    else
        prescribed_part<3><<<gn, kVT, 0, st>>>(w->nn, m->node_mask, u, uc);
    FEM_TRY(femi::run_op(m, FEM_F64, fem::OP_RESIDUAL, u, nullptr, r, nullptr, 0u, st, nullptr));
    dot_kernel<double, double><<<gd, kVT, 0, st>>>(w->nd, uc, r, w->dot, w->partial);
    CUDA_TRY(cudaMemcpyAsync(c_dev, &w->dot->value, sizeof(double), cudaMemcpyDeviceToDevice, st));
    // 2. right-hand side K_fc u_c: an HVP with u_c as the direction, rows of
    // the free DOFs only
    FEM_TRY(femi::run_op(m, FEM_F64, fem::OP_HVP, u, uc, rhs, nullptr, (unsigned)FEM_MASK_OUT, st, nullptr));
    // 3. adjoint solve K_ff lam = K_fc u_c (the PCG of the Newton step).  With
    // an FP32 PCG the solve is refined in FP64 (mixed-precision iterative
    // refinement): the FP64 residual rhs - M K M lam of the current lam is
    // solved for a correction by the FP32 PCG to a modest tolerance, and added;
    // the FP32 solve alone stalls near its own rounding level, far above
    // rtol on fine meshes.
    fem_newton_opts o;
    fem_newton_default_opts(&o);
    o.cg_dtype = cg_dtype;
    fem_newton_stats stats{};
    Stepper stepper(m, o, &stats, st);
    fem_status err = FEM_OK;
    int64_t it_total = 0;
    auto solve = [&](const double* b, double* x, double tol) -> fem_status {
        int64_t it = 0;
        const int rc = stepper.tangent_solve(u, b, x, tol, &it, &err);
        it_total += it;
        if (err != FEM_OK) return err;
        if (rc == 5) return fail(FEM_ERR_NOT_SPD, "fem_compliance_gradient: a nodal diagonal block is not SPD");
        if (rc == 2) return fail(FEM_ERR_NEG_CURVATURE, "fem_compliance_gradient: p^T K p <= 0 in the adjoint solve");
        if (rc == 3) return fail(FEM_ERR_NOT_CONVERGED, "fem_compliance_gradient: adjoint iteration cap reached");
        return FEM_OK;
    };
    if (cg_dtype == FEM_F64) {
        FEM_TRY(solve(rhs, lam, rtol));
    } else {
        constexpr double kInner = 1e-4;  // FP32 PCG tolerance of each correction
        constexpr int kMaxRefine = 8;
        double* res = r;  // the residual vector is free again once c is copied out
        if (!w->adj) FEM_TRY(dalloc(w, &w->adj, (size_t)w->nd));
        double* dlam = w->adj;
        double bb = 0.0;
        dot_kernel<double, double><<<gd, kVT, 0, st>>>(w->nd, rhs, rhs, w->dot, w->partial);
        CUDA_TRY(cudaMemcpyAsync(&w->h->dot, w->dot, sizeof(DotState), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        bb = w->h->dot.value;
        FEM_TRY(solve(rhs, lam, kInner));
        for (int k = 0; k < kMaxRefine; ++k) {
            // res = rhs - M K M lam (FP64)
            FEM_TRY(femi::run_op(m, FEM_F64, fem::OP_HVP, u, lam, res, nullptr, (unsigned)FEM_MASK_BOTH, st, nullptr));
            residual_update<<<gd, kVT, 0, st>>>(w->nd, rhs, res);
            dot_kernel<double, double><<<gd, kVT, 0, st>>>(w->nd, res, res, w->dot, w->partial);
            CUDA_TRY(cudaMemcpyAsync(&w->h->dot, w->dot, sizeof(DotState), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            const double rr = w->h->dot.value;
            if (!(rr > rtol * rtol * bb)) break;
            FEM_TRY(solve(res, dlam, kInner));
            add_into<<<gd, kVT, 0, st>>>(w->nd, dlam, lam);
        }
    }
    if (iters) *iters = it_total;
    // 4. a = u_c - lam; dc/dmu_e = a^T (dr_e/dmu_e + ratio dr_e/dlambda_e)
    const bool f32 = vjp_dtype == FEM_F32;
    adjoint_weights<<<gd, kVT, 0, st>>>(w->nd, uc, lam, uc, f32 ? w->du32 : nullptr);
    if (f32) {
        to_f32<<<gd, kVT, 0, st>>>(w->nd, u, w->u32);
        FEM_TRY(fem_param_vjp(m, FEM_F32, w->u32, w->du32, dmu, w->glam, st));
    } else {
        FEM_TRY(fem_param_vjp(m, FEM_F64, u, uc, dmu, w->glam, st));
    }
    tied_moduli<<<grid_for(m->info.n_elems), kVT, 0, st>>>(m->info.n_elems, dmu, w->glam, ratio);
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // extern "C"
