// Tile kernels of the energy-based FEM hot path (sm_103a).
//
// One CTA owns one tile (see fem_plan.h).  It stages the tile's nodal data
// in shared memory, runs the tile's rounds (warp w takes rounds w, w+4, ...;
// one element per lane; the elements of a round share no node), accumulates
// nodal results into its warp's private shared-memory copy, combines the
// copies in warp order and writes: private nodes directly, shared nodes as
// a partial into their fixed slot.  The last tile to finish a shared node
// (an integer arrival counter per node) sums its slots in slot order.  Every
// sum therefore has a fixed order: results are bitwise reproducible and no
// floating-point atomic is used.
//
// Per element (Algorithm 1 of arXiv 2602.12365): gather nodal values, form
// H = grad u = sum_a u_a (x) grad N_a and F = I + H, evaluate the
// compressible Neo-Hookean density / stress / tangent action, multiply by
// w_q det J and scatter.  P1 elements read precomputed grad N_a and w det J
// from a per-round record; Q1 hexahedra rebuild J from the staged nodal
// coordinates at each of the 2x2x2 Gauss points.
//
// FP32 accuracy: J - 1 is formed from the invariants of H and F^-T - I from
// the cofactor identity cof(I + H) = (1 + tr H) I - H^T + cof(H), so no
// quantity near 1 is ever subtracted from 1; differences u_a - u_ref are taken
// before the gradient sums.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr int kSpinLimit = 1 << 22;

enum Op { OP_ENERGY = 0, OP_RESIDUAL = 1, OP_HVP = 2, OP_BLOCKDIAG = 3, OP_PVJP = 4 };

template <int ET>
struct ElemT;
template <>
struct ElemT<0> {  // P1 triangle, plane strain
    static constexpr int D = 2, NEN = 3, NQ = 1, PAD = 4, NG = 5, VW = 2;
};
template <>
struct ElemT<1> {  // P1 tetrahedron
    static constexpr int D = 3, NEN = 4, NQ = 1, PAD = 4, NG = 10, VW = 4;
};
template <>
struct ElemT<2> {  // Q1 hexahedron, 2x2x2 Gauss
    static constexpr int D = 3, NEN = 8, NQ = 8, PAD = 8, NG = 0, VW = 4;
};

// shared-memory layout (bytes), identical on host and device
struct SmemLayout {
    int off_u, off_v, off_x, off_acc, off_mask, off_red, total, aw;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int et, int tsize, int op, int nl) {
    SmemLayout L;
    int D = et == 0 ? 2 : 3;
    int VW = D == 2 ? 2 : 4;
    int vec = VW * tsize;
    L.aw = (op == OP_BLOCKDIAG) ? (D == 2 ? 4 : 6) : VW;
    bool need_v = (op == OP_HVP || op == OP_PVJP);
    bool need_acc = (op == OP_RESIDUAL || op == OP_HVP || op == OP_BLOCKDIAG);
    int o = 0;
    L.off_u = o;
    o = align16(o + nl * vec);
    L.off_v = o;
    if (need_v) o = align16(o + nl * vec);
    L.off_x = o;
    if (et == 2) o = align16(o + nl * vec);
    L.off_acc = o;
    if (need_acc) o = align16(o + kWarps * nl * L.aw * tsize);
    L.off_mask = o;
    o = align16(o + nl);
    L.off_red = o;
    o = align16(o + kWarps * 4 * 8 + 16);
    L.total = o;
    return L;
}

struct KParams {
    // plan
    const int32_t* tile_round_ptr;
    const int64_t* tile_node_ptr;
    const int32_t* node_gid;
    const int32_t* node_slot;
    const uint8_t* round_nvalid;
    const int32_t* round_elem;
    const uint8_t* rec;
    int64_t rec_bytes;
    int geom_off;
    int mat_off;  // -1: uniform moduli
    const int32_t* slot_owner;
    const int32_t* shared_gid;
    const int64_t* shared_slot_ptr;
    int32_t* shared_count;
    const int32_t* orphans;
    int n_orphans;
    const uint8_t* node_mask;
    const void* X;  // Q1: nodal coordinates [n_nodes][3] in the kernel's dtype
    int n_tiles;
    double mu0, lam0;
    // workspace
    void* partial;
    double* tile_red;
    unsigned* tile_counter;
    int* status;
    // call
    const void* u;
    const void* v;
    void* out;
    double* out_scalar;
    double* out_mu;
    double* out_lam;
    unsigned flags;
};

// ---------------------------------------------------------------------------
// scalar helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
__device__ __forceinline__ double log1p_(double x) { return log1p(x); }
__device__ __forceinline__ bool finite_(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_(double x) { return isfinite(x); }

template <typename T>
__device__ __forceinline__ T ldg_(const T* p) {
    return __ldg(p);
}

// Nodal vectors in shared memory: VW-wide, 16-byte aligned for 3D FP32.
template <int VW, typename T>
__device__ __forceinline__ void lds_vec(const T* base, int i, T* out) {
    if constexpr (VW == 4 && sizeof(T) == 4) {
        float4 t = reinterpret_cast<const float4*>(base)[i];
        out[0] = t.x;
        out[1] = t.y;
        out[2] = t.z;
    } else if constexpr (VW == 2 && sizeof(T) == 4) {
        float2 t = reinterpret_cast<const float2*>(base)[i];
        out[0] = t.x;
        out[1] = t.y;
    } else if constexpr (VW == 4) {
        double2 a = reinterpret_cast<const double2*>(base)[2 * i];
        double2 b = reinterpret_cast<const double2*>(base)[2 * i + 1];
        out[0] = a.x;
        out[1] = a.y;
        out[2] = b.x;
    } else {
        double2 a = reinterpret_cast<const double2*>(base)[i];
        out[0] = a.x;
        out[1] = a.y;
    }
}

template <int VW, typename T>
__device__ __forceinline__ void sts_vec(T* base, int i, const T* in) {
    if constexpr (VW == 4 && sizeof(T) == 4) {
        reinterpret_cast<float4*>(base)[i] = make_float4(in[0], in[1], in[2], 0.f);
    } else if constexpr (VW == 2 && sizeof(T) == 4) {
        reinterpret_cast<float2*>(base)[i] = make_float2(in[0], in[1]);
    } else if constexpr (VW == 4) {
        reinterpret_cast<double2*>(base)[2 * i] = make_double2(in[0], in[1]);
        reinterpret_cast<double2*>(base)[2 * i + 1] = make_double2(in[2], 0.0);
    } else {
        reinterpret_cast<double2*>(base)[i] = make_double2(in[0], in[1]);
    }
}

// acc[i] += f (read-modify-write of one nodal accumulator)
template <int VW, int D, typename T>
__device__ __forceinline__ void rmw_vec(T* base, int i, const T* f) {
    T cur[4];
    lds_vec<VW, T>(base, i, cur);
#pragma unroll
    for (int k = 0; k < D; ++k) cur[k] += f[k];
    sts_vec<VW, T>(base, i, cur);
}

// ---------------------------------------------------------------------------
// Neo-Hookean kinematics from H = grad u
// ---------------------------------------------------------------------------
template <int D, typename T>
struct Kin {
    T G[D][D];  // F^-T - I
    T lnJ;
    T trH, HH;  // tr H, H:H
    bool ok;    // J > 0
};

template <int D, typename T>
__device__ __forceinline__ void kinematics(const T (&H)[D][D], Kin<D, T>& k) {
    k.trH = 0;
    k.HH = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        k.trH += H[i][i];
#pragma unroll
        for (int j = 0; j < D; ++j) k.HH = fma(H[i][j], H[i][j], k.HH);
    }
    if constexpr (D == 2) {
        T detH = H[0][0] * H[1][1] - H[0][1] * H[1][0];
        T Jm1 = k.trH + detH;
        T J = T(1) + Jm1;
        k.ok = J > T(0);
        T rJ = rcp_(J);
        // cof(F) - J I = -det(H) I - H^T
        k.G[0][0] = (-detH - H[0][0]) * rJ;
        k.G[0][1] = -H[1][0] * rJ;
        k.G[1][0] = -H[0][1] * rJ;
        k.G[1][1] = (-detH - H[1][1]) * rJ;
        k.lnJ = k.ok ? log1p_(Jm1) : T(0);
    } else {
        T c[3][3];
        c[0][0] = H[1][1] * H[2][2] - H[1][2] * H[2][1];
        c[0][1] = H[1][2] * H[2][0] - H[1][0] * H[2][2];
        c[0][2] = H[1][0] * H[2][1] - H[1][1] * H[2][0];
        c[1][0] = H[0][2] * H[2][1] - H[0][1] * H[2][2];
        c[1][1] = H[0][0] * H[2][2] - H[0][2] * H[2][0];
        c[1][2] = H[0][1] * H[2][0] - H[0][0] * H[2][1];
        c[2][0] = H[0][1] * H[1][2] - H[0][2] * H[1][1];
        c[2][1] = H[0][2] * H[1][0] - H[0][0] * H[1][2];
        c[2][2] = H[0][0] * H[1][1] - H[0][1] * H[1][0];
        T I2 = c[0][0] + c[1][1] + c[2][2];
        T detH = H[0][0] * c[0][0] + H[0][1] * c[0][1] + H[0][2] * c[0][2];
        T s = I2 + detH;
        T Jm1 = k.trH + s;
        T J = T(1) + Jm1;
        k.ok = J > T(0);
        T rJ = rcp_(J);
        // cof(F) - J I = cof(H) - H^T - (I2 + det H) I
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) k.G[i][j] = (c[i][j] - H[j][i] - (i == j ? s : T(0))) * rJ;
        k.lnJ = k.ok ? log1p_(Jm1) : T(0);
    }
}

// psi = mu (tr H + H:H/2 - ln J) + lam/2 ln^2 J  (= mu/2 (I1-3) - mu lnJ + lam/2 ln^2 J)
// scale = mu (I1/2 + |ln J|) + lam/2 ln^2 J, I1 = 3 + 2 tr H + H:H
template <int D, typename T>
__device__ __forceinline__ void density(const Kin<D, T>& k, T mu, T lam, T& psi, T& scale) {
    T l2 = T(0.5) * lam * k.lnJ * k.lnJ;
    psi = mu * (k.trH + T(0.5) * k.HH - k.lnJ) + l2;
    T I1 = T(3) + T(2) * k.trH + k.HH;
    scale = mu * (T(0.5) * I1 + fabs(k.lnJ)) + l2;
}

// P = mu (F - F^-T) + lam ln J F^-T = mu (H - G) + lam lnJ (I + G)
template <int D, typename T>
__device__ __forceinline__ void stress(const T (&H)[D][D], const Kin<D, T>& k, T mu, T lam,
                                       T (&P)[D][D]) {
    T ll = lam * k.lnJ;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j)
            P[i][j] = mu * (H[i][j] - k.G[i][j]) + ll * (k.G[i][j] + (i == j ? T(1) : T(0)));
}

// dP = mu dF + (mu - lam lnJ) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T
template <int D, typename T>
__device__ __forceinline__ void tangent(const T (&dF)[D][D], const Kin<D, T>& k, T mu, T lam,
                                        T (&dP)[D][D]) {
    T FiT[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) FiT[i][j] = k.G[i][j] + (i == j ? T(1) : T(0));
    T trA = 0;  // tr(F^-1 dF) = F^-T : dF
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) trA = fma(FiT[i][j], dF[i][j], trA);
    T M[D][D];  // dF^T F^-T
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T s = 0;
#pragma unroll
            for (int l = 0; l < D; ++l) s = fma(dF[l][a], FiT[l][j], s);
            M[a][j] = s;
        }
    T c1 = mu - lam * k.lnJ;
    T c2 = lam * trA;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T B = 0;  // (F^-T M)_ij
#pragma unroll
            for (int a = 0; a < D; ++a) B = fma(FiT[i][a], M[a][j], B);
            dP[i][j] = mu * dF[i][j] + c1 * B + c2 * FiT[i][j];
        }
}

// ---------------------------------------------------------------------------
// Q1 reference gradients at the 2x2x2 Gauss points (compile-time constants)
// ---------------------------------------------------------------------------
constexpr double kGauss = 0.57735026918962576451;  // 1/sqrt(3)

__host__ __device__ constexpr int hex_sign(int a, int j) {
    // VTK_HEXAHEDRON: (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1)
    return j == 0 ? (((a & 3) == 1 || (a & 3) == 2) ? 1 : -1)
                  : (j == 1 ? (((a & 3) >= 2) ? 1 : -1) : ((a >= 4) ? 1 : -1));
}

__host__ __device__ constexpr double hex_xi(int q, int j) {
    return ((q >> j) & 1) ? kGauss : -kGauss;
}

// d N_a / d xi_j at Gauss point q
__host__ __device__ constexpr double hex_dN(int a, int q, int j) {
    double f0 = 1.0 + hex_sign(a, 0) * hex_xi(q, 0);
    double f1 = 1.0 + hex_sign(a, 1) * hex_xi(q, 1);
    double f2 = 1.0 + hex_sign(a, 2) * hex_xi(q, 2);
    return j == 0 ? 0.125 * hex_sign(a, 0) * f1 * f2
                  : (j == 1 ? 0.125 * hex_sign(a, 1) * f0 * f2 : 0.125 * hex_sign(a, 2) * f0 * f1);
}

// ---------------------------------------------------------------------------
// per-element work.  `ue`, `ve`, `xe` hold the gathered nodal vectors; results
// go to f[NEN][AW] (nodal contributions) and the scalar accumulators.
// ---------------------------------------------------------------------------
template <int D, typename T>
__device__ __forceinline__ void outer_sum(const T (*du)[D], const T (*g)[D], int n, T (&H)[D][D]) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) H[i][j] = 0;
    for (int a = 0; a < n; ++a)
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) H[i][j] = fma(du[a][i], g[a][j], H[i][j]);
}

struct ScalarAcc {
    double s0 = 0, s1 = 0;
    int ninv = 0;
};

// Quadrature-point work common to P1 and Q1: given H (and dF), the gradients
// g[a] of the NEN-1 non-reference nodes and wdJ, produce the contributions
// f[a] for those nodes (the reference node gets minus their sum).
template <int OP, int D, int NM1, typename T>
__device__ __forceinline__ void qp_work(const T (&H)[D][D], const T (&dF)[D][D], const T (&g)[NM1][D],
                                        T wdJ, T mu, T lam, T (&f)[NM1 + 1][6], ScalarAcc& acc,
                                        const T (&da)[D][D], double& gmu, double& glam, bool& inv) {
    Kin<D, T> k;
    kinematics<D, T>(H, k);
    if (!k.ok) {
        inv = true;
        acc.ninv++;
        return;
    }
    if constexpr (OP == OP_ENERGY) {
        T psi, sc;
        density<D, T>(k, mu, lam, psi, sc);
        acc.s0 += (double)(wdJ * psi);
        acc.s1 += (double)(wdJ * sc);
    } else if constexpr (OP == OP_RESIDUAL || OP == OP_HVP) {
        T P[D][D];
        if constexpr (OP == OP_RESIDUAL) {
            stress<D, T>(H, k, mu, lam, P);
        } else {
            tangent<D, T>(dF, k, mu, lam, P);
            T s = 0;
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) s = fma(P[i][j], dF[i][j], s);
            acc.s0 += (double)(wdJ * s);
        }
#pragma unroll
        for (int a = 0; a < NM1; ++a)
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T s = 0;
#pragma unroll
                for (int j = 0; j < D; ++j) s = fma(P[i][j], g[a][j], s);
                f[a][i] = fma(wdJ, s, f[a][i]);
            }
    } else if constexpr (OP == OP_BLOCKDIAG) {
        // K_aa = wdJ [mu |g0|^2 I + (mu - lam lnJ + lam) gp gp^T], gp = F^-T g0
        T c = wdJ * (mu + lam * (T(1) - k.lnJ));
        T m = wdJ * mu;
#pragma unroll
        for (int a = 0; a <= NM1; ++a) {
            T g0[D];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                if (a < NM1) {
                    g0[j] = g[a][j];
                } else {
                    T s = 0;
#pragma unroll
                    for (int b = 0; b < NM1; ++b) s -= g[b][j];
                    g0[j] = s;
                }
            }
            T gp[D];
            T n2 = 0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T s = g0[i];
#pragma unroll
                for (int j = 0; j < D; ++j) s = fma(k.G[i][j], g0[j], s);
                gp[i] = s;
                n2 = fma(g0[i], g0[i], n2);
            }
            T mn = m * n2;
            if constexpr (D == 3) {
                f[a][0] += mn + c * gp[0] * gp[0];
                f[a][1] += mn + c * gp[1] * gp[1];
                f[a][2] += mn + c * gp[2] * gp[2];
                f[a][3] += c * gp[0] * gp[1];
                f[a][4] += c * gp[0] * gp[2];
                f[a][5] += c * gp[1] * gp[2];
            } else {
                f[a][0] += mn + c * gp[0] * gp[0];
                f[a][1] += mn + c * gp[1] * gp[1];
                f[a][2] += c * gp[0] * gp[1];
            }
        }
    } else if constexpr (OP == OP_PVJP) {
        // dP/dmu : grad a = (H - G) : grad a ; dP/dlam : grad a = lnJ (I + G) : grad a
        T sm = 0, sl = 0;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                sm = fma(H[i][j] - k.G[i][j], da[i][j], sm);
                sl = fma(k.G[i][j] + (i == j ? T(1) : T(0)), da[i][j], sl);
            }
        gmu += (double)(wdJ * sm);
        glam += (double)(wdJ * k.lnJ * sl);
    }
}

// ---------------------------------------------------------------------------
// the tile kernel
// ---------------------------------------------------------------------------
template <int ET, typename T, int OP>
__global__ void __launch_bounds__(kThreads) tile_kernel(const KParams p) {
    using E = ElemT<ET>;
    constexpr int D = E::D, NEN = E::NEN, VW = E::VW, NM1 = NEN - 1;
    constexpr bool kNeedV = (OP == OP_HVP || OP == OP_PVJP);
    constexpr bool kNeedAcc = (OP == OP_RESIDUAL || OP == OP_HVP || OP == OP_BLOCKDIAG);
    extern __shared__ __align__(16) unsigned char smem[];

    const int tile = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n0 = p.tile_node_ptr[tile];
    const int nl = (int)(p.tile_node_ptr[tile + 1] - n0);
    const SmemLayout L = smem_layout(ET, (int)sizeof(T), OP, nl);
    const int AW = L.aw;
    T* sU = reinterpret_cast<T*>(smem + L.off_u);
    T* sV = reinterpret_cast<T*>(smem + L.off_v);
    T* sX = reinterpret_cast<T*>(smem + L.off_x);
    T* sAcc = reinterpret_cast<T*>(smem + L.off_acc);
    uint8_t* sMask = smem + L.off_mask;
    double* sRed = reinterpret_cast<double*>(smem + L.off_red);
    int* sFlag = reinterpret_cast<int*>(smem + L.off_red + kWarps * 4 * 8);

    const T* gu = static_cast<const T*>(p.u);
    const T* gv = static_cast<const T*>(p.v);
    int flags_local = 0;

    // 1. stage the tile's nodes
    for (int i = tid; i < nl; i += kThreads) {
        const int g = p.node_gid[n0 + i];
        const uint8_t m = p.node_mask[g];
        T t[4] = {0, 0, 0, 0};
        bool fin = true;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            t[k] = gu[(int64_t)g * D + k];
            fin = fin && finite_(t[k]);
        }
        sts_vec<VW, T>(sU, i, t);
        if constexpr (kNeedV) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                T x = gv[(int64_t)g * D + k];
                if (OP == OP_HVP && (p.flags & 2u) && ((m >> k) & 1)) x = T(0);
                fin = fin && finite_(x);
                t[k] = x;
            }
            sts_vec<VW, T>(sV, i, t);
        }
        if constexpr (ET == 2) {
            const T* gx = static_cast<const T*>(p.X);
#pragma unroll
            for (int k = 0; k < D; ++k) t[k] = gx[(int64_t)g * D + k];
            sts_vec<VW, T>(sX, i, t);
        }
        if (!fin) flags_local |= 2;
        sMask[i] = m;
        if constexpr (kNeedAcc) {
            for (int w = 0; w < kWarps; ++w)
                for (int k = 0; k < AW; ++k) sAcc[((int64_t)w * nl + i) * AW + k] = T(0);
        }
    }
    if (tid == 0) *sFlag = 0;
    __syncthreads();

    // 2. rounds
    ScalarAcc acc;
    T* myAcc = sAcc + (int64_t)warp * nl * AW;
    const int r_begin = p.tile_round_ptr[tile], r_end = p.tile_round_ptr[tile + 1];
    bool inv = false;
    for (int r = r_begin + warp; r < r_end; r += kWarps) {
        const int nv = p.round_nvalid[r];
        const uint8_t* rec = p.rec + (int64_t)r * p.rec_bytes;
        if (lane < nv) {
            int cn[NEN];
            if constexpr (E::PAD == 4) {
                uint2 w = __ldg(reinterpret_cast<const uint2*>(rec) + lane);
                cn[0] = w.x & 0xffff;
                cn[1] = w.x >> 16;
                cn[2] = w.y & 0xffff;
                if constexpr (NEN == 4) cn[3] = w.y >> 16;
            } else {
                uint4 w = __ldg(reinterpret_cast<const uint4*>(rec) + lane);
                cn[0] = w.x & 0xffff;
                cn[1] = w.x >> 16;
                cn[2] = w.y & 0xffff;
                cn[3] = w.y >> 16;
                cn[4] = w.z & 0xffff;
                cn[5] = w.z >> 16;
                cn[6] = w.w & 0xffff;
                cn[7] = w.w >> 16;
            }
            T mu = (T)p.mu0, lam = (T)p.lam0;
            if (p.mat_off >= 0) {
                const T* mat = reinterpret_cast<const T*>(rec + p.mat_off);
                mu = ldg_(mat + lane);
                lam = ldg_(mat + 32 + lane);
            }
            // gather
            T ue[NEN][D], ve[NEN][D];
#pragma unroll
            for (int a = 0; a < NEN; ++a) {
                T t[4];
                lds_vec<VW, T>(sU, cn[a], t);
#pragma unroll
                for (int k = 0; k < D; ++k) ue[a][k] = t[k];
                if constexpr (kNeedV) {
                    lds_vec<VW, T>(sV, cn[a], t);
#pragma unroll
                    for (int k = 0; k < D; ++k) ve[a][k] = t[k];
                }
            }
            T f[NEN][6];
#pragma unroll
            for (int a = 0; a < NEN; ++a)
#pragma unroll
                for (int k = 0; k < 6; ++k) f[a][k] = 0;
            double gmu = 0, glam = 0;

            if constexpr (ET != 2) {
                // P1: reference node = last; grad N_a (a < NEN-1) and w detJ precomputed
                const T* geom = reinterpret_cast<const T*>(rec + p.geom_off);
                T g[NM1][D];
#pragma unroll
                for (int a = 0; a < NM1; ++a)
#pragma unroll
                    for (int k = 0; k < D; ++k) g[a][k] = ldg_(geom + (a * D + k) * 32 + lane);
                const T wdJ = ldg_(geom + (E::NG - 1) * 32 + lane);
                T du[NM1][D], dv[NM1][D];
#pragma unroll
                for (int a = 0; a < NM1; ++a)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        du[a][k] = ue[a][k] - ue[NM1][k];
                        if constexpr (kNeedV) dv[a][k] = ve[a][k] - ve[NM1][k];
                    }
                T H[D][D], dF[D][D] = {};
                outer_sum<D, T>(du, g, NM1, H);
                if constexpr (kNeedV) outer_sum<D, T>(dv, g, NM1, dF);
                T fq[NM1 + 1][6];
#pragma unroll
                for (int a = 0; a <= NM1; ++a)
#pragma unroll
                    for (int k = 0; k < 6; ++k) fq[a][k] = 0;
                qp_work<OP, D, NM1, T>(H, dF, g, wdJ, mu, lam, fq, acc, dF, gmu, glam, inv);
                if constexpr (OP == OP_RESIDUAL || OP == OP_HVP) {
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        T s = 0;
#pragma unroll
                        for (int a = 0; a < NM1; ++a) {
                            f[a][k] = fq[a][k];
                            s -= fq[a][k];
                        }
                        f[NM1][k] = s;
                    }
                } else if constexpr (OP == OP_BLOCKDIAG) {
#pragma unroll
                    for (int a = 0; a <= NM1; ++a)
#pragma unroll
                        for (int k = 0; k < 6; ++k) f[a][k] = fq[a][k];
                }
            } else {
                // Q1: reference node 0; J rebuilt at each Gauss point
                T dx[NM1][D], du[NM1][D], dv[NM1][D];
                {
                    T x0[4];
                    lds_vec<VW, T>(sX, cn[0], x0);
#pragma unroll
                    for (int a = 1; a < NEN; ++a) {
                        T t[4];
                        lds_vec<VW, T>(sX, cn[a], t);
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            dx[a - 1][k] = t[k] - x0[k];
                            du[a - 1][k] = ue[a][k] - ue[0][k];
                            if constexpr (kNeedV) dv[a - 1][k] = ve[a][k] - ve[0][k];
                        }
                    }
                }
                T fr[NEN][6];  // contributions of nodes 1..7, then node 0 (block diagonal)
#pragma unroll
                for (int a = 0; a < NEN; ++a)
#pragma unroll
                    for (int k = 0; k < 6; ++k) fr[a][k] = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    T gr[NM1][D];  // reference gradients of nodes 1..7
#pragma unroll
                    for (int a = 0; a < NM1; ++a)
#pragma unroll
                        for (int j = 0; j < D; ++j) gr[a][j] = (T)hex_dN(a + 1, q, j);
                    T Jm[D][D];
                    outer_sum<D, T>(dx, gr, NM1, Jm);
                    // inverse of J by cofactors
                    T c00 = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
                    T c01 = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
                    T c02 = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
                    T detJ = Jm[0][0] * c00 + Jm[0][1] * c01 + Jm[0][2] * c02;
                    T rd = rcp_(detJ);
                    T Ji[3][3];  // J^-1
                    Ji[0][0] = c00 * rd;
                    Ji[1][0] = c01 * rd;
                    Ji[2][0] = c02 * rd;
                    Ji[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) * rd;
                    Ji[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) * rd;
                    Ji[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) * rd;
                    Ji[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) * rd;
                    Ji[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) * rd;
                    Ji[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) * rd;
                    // physical gradients g_a = J^-T grad N^_a
                    T g[NM1][D];
#pragma unroll
                    for (int a = 0; a < NM1; ++a)
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            T s = 0;
#pragma unroll
                            for (int j = 0; j < D; ++j) s = fma(Ji[j][i], gr[a][j], s);
                            g[a][i] = s;
                        }
                    T H[D][D], dF[D][D] = {};
                    outer_sum<D, T>(du, g, NM1, H);
                    if constexpr (kNeedV) outer_sum<D, T>(dv, g, NM1, dF);
                    qp_work<OP, D, NM1, T>(H, dF, g, detJ, mu, lam, fr, acc, dF, gmu, glam, inv);
                }
                if constexpr (OP == OP_RESIDUAL || OP == OP_HVP) {
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        T s = 0;
#pragma unroll
                        for (int a = 0; a < NM1; ++a) {
                            f[a + 1][k] = fr[a][k];
                            s -= fr[a][k];
                        }
                        f[0][k] = s;
                    }
                } else if constexpr (OP == OP_BLOCKDIAG) {
                    // qp_work put nodes 1..7 in rows 0..6 and node 0 in row 7
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        f[0][k] = fr[NM1][k];
#pragma unroll
                        for (int a = 0; a < NM1; ++a) f[a + 1][k] = fr[a][k];
                    }
                }
            }

            if constexpr (OP == OP_PVJP) {
                const int e = p.round_elem[(int64_t)r * 32 + lane];
                if (p.out_mu) p.out_mu[e] = gmu;
                if (p.out_lam) p.out_lam[e] = glam;
            }
            if constexpr (OP == OP_RESIDUAL || OP == OP_HVP) {
#pragma unroll
                for (int a = 0; a < NEN; ++a) rmw_vec<VW, D, T>(myAcc, cn[a], f[a]);
            } else if constexpr (OP == OP_BLOCKDIAG) {
#pragma unroll
                for (int a = 0; a < NEN; ++a)
                    for (int k = 0; k < AW; ++k) myAcc[cn[a] * AW + k] += f[a][k];
            }
            (void)gmu;
            (void)glam;
        }
        __syncwarp();
    }
    if (inv) flags_local |= 1;

    // 3. block reductions of the scalar accumulators (fixed order)
    if constexpr (OP == OP_ENERGY || OP == OP_HVP) {
        double s0 = acc.s0, s1 = acc.s1, s2 = (double)acc.ninv;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            sRed[warp * 4 + 0] = s0;
            sRed[warp * 4 + 1] = s1;
            sRed[warp * 4 + 2] = s2;
        }
    }
    {
        int wf = __reduce_or_sync(0xffffffffu, flags_local);
        if (lane == 0 && wf) atomicOr(sFlag, wf);
    }
    __syncthreads();

    // 4. combine the warp copies and write nodal results
    if constexpr (kNeedAcc) {
        T* part = static_cast<T*>(p.partial);
        T* out = static_cast<T*>(p.out);
        int wflag = 0;
        for (int i = tid; i < nl; i += kThreads) {
            T s[6] = {0, 0, 0, 0, 0, 0};
            for (int w = 0; w < kWarps; ++w)
                for (int k = 0; k < AW; ++k) s[k] += sAcc[((int64_t)w * nl + i) * AW + k];
            const int slot = p.node_slot[n0 + i];
            const int g = p.node_gid[n0 + i];
            if (slot < 0) {
                const uint8_t m = sMask[i];
                if constexpr (OP == OP_BLOCKDIAG) {
                    T Dm[D][D];
                    if constexpr (D == 3) {
                        Dm[0][0] = s[0]; Dm[1][1] = s[1]; Dm[2][2] = s[2];
                        Dm[0][1] = Dm[1][0] = s[3];
                        Dm[0][2] = Dm[2][0] = s[4];
                        Dm[1][2] = Dm[2][1] = s[5];
                    } else {
                        Dm[0][0] = s[0]; Dm[1][1] = s[1];
                        Dm[0][1] = Dm[1][0] = s[2];
                    }
                    for (int a = 0; a < D; ++a)
                        for (int b = 0; b < D; ++b) {
                            T x = Dm[a][b];
                            if (((m >> a) & 1) || ((m >> b) & 1)) x = (a == b) ? T(1) : T(0);
                            if (!finite_(x)) wflag |= 2;
                            out[((int64_t)g * D + a) * D + b] = x;
                        }
                } else {
                    for (int k = 0; k < D; ++k) {
                        T x = s[k];
                        if ((p.flags & 1u) && ((m >> k) & 1)) x = T(0);
                        if (!finite_(x)) wflag |= 2;
                        out[(int64_t)g * D + k] = x;
                    }
                }
            } else {
                for (int k = 0; k < AW; ++k) part[(int64_t)slot * AW + k] = s[k];
            }
        }
        if (wflag) atomicOr(sFlag, wflag);
        __threadfence();
        __syncthreads();
        // last arriver of each shared node sums its slots in slot order
        for (int i = tid; i < nl; i += kThreads) {
            const int slot = p.node_slot[n0 + i];
            if (slot < 0) continue;
            const int sid = p.slot_owner[slot];
            const int64_t s0 = p.shared_slot_ptr[sid], s1 = p.shared_slot_ptr[sid + 1];
            const int old = atomicAdd(&p.shared_count[sid], 1);
            if (old != (int)(s1 - s0) - 1) continue;
            __threadfence();
            T s[6] = {0, 0, 0, 0, 0, 0};
            for (int64_t q = s0; q < s1; ++q)
                for (int k = 0; k < AW; ++k) s[k] += __ldcg(part + q * AW + k);
            p.shared_count[sid] = 0;
            const int g = p.node_gid[n0 + i];
            const uint8_t m = sMask[i];
            int fl = 0;
            if constexpr (OP == OP_BLOCKDIAG) {
                T Dm[D][D];
                if constexpr (D == 3) {
                    Dm[0][0] = s[0]; Dm[1][1] = s[1]; Dm[2][2] = s[2];
                    Dm[0][1] = Dm[1][0] = s[3];
                    Dm[0][2] = Dm[2][0] = s[4];
                    Dm[1][2] = Dm[2][1] = s[5];
                } else {
                    Dm[0][0] = s[0]; Dm[1][1] = s[1];
                    Dm[0][1] = Dm[1][0] = s[2];
                }
                for (int a = 0; a < D; ++a)
                    for (int b = 0; b < D; ++b) {
                        T x = Dm[a][b];
                        if (((m >> a) & 1) || ((m >> b) & 1)) x = (a == b) ? T(1) : T(0);
                        if (!finite_(x)) fl |= 2;
                        out[((int64_t)g * D + a) * D + b] = x;
                    }
            } else {
                for (int k = 0; k < D; ++k) {
                    T x = s[k];
                    if ((p.flags & 1u) && ((m >> k) & 1)) x = T(0);
                    if (!finite_(x)) fl |= 2;
                    out[(int64_t)g * D + k] = x;
                }
            }
            if (fl) atomicOr(p.status, fl);
        }
        // nodes that belong to no element
        if (tile == 0) {
            for (int i = tid; i < p.n_orphans; i += kThreads) {
                const int g = p.orphans[i];
                if constexpr (OP == OP_BLOCKDIAG) {
                    for (int a = 0; a < D; ++a)
                        for (int b = 0; b < D; ++b) out[((int64_t)g * D + a) * D + b] = (a == b) ? T(1) : T(0);
                } else {
                    for (int k = 0; k < D; ++k) out[(int64_t)g * D + k] = T(0);
                }
            }
        }
    }

    // 5. tile partial of the scalars; the last tile reduces them in tile order
    if (OP == OP_ENERGY || (OP == OP_HVP && p.out_scalar != nullptr)) {
        __shared__ int s_last;
        if (tid == 0) {
            double a0 = 0, a1 = 0, a2 = 0;
            for (int w = 0; w < kWarps; ++w) {
                a0 += sRed[w * 4 + 0];
                a1 += sRed[w * 4 + 1];
                a2 += sRed[w * 4 + 2];
            }
            p.tile_red[(int64_t)tile * 4 + 0] = a0;
            p.tile_red[(int64_t)tile * 4 + 1] = a1;
            p.tile_red[(int64_t)tile * 4 + 2] = a2;
            __threadfence();
            const unsigned old = atomicAdd(p.tile_counter, 1u);
            s_last = (old == (unsigned)p.n_tiles - 1u);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            // per-thread Neumaier sums over a fixed strided subset, then a
            // fixed combination order
            double sum0 = 0, c0 = 0, sum1 = 0, c1 = 0, cnt = 0;
            for (int t = tid; t < p.n_tiles; t += kThreads) {
                const double x0 = __ldcg(p.tile_red + (int64_t)t * 4 + 0);
                const double x1 = __ldcg(p.tile_red + (int64_t)t * 4 + 1);
                cnt += __ldcg(p.tile_red + (int64_t)t * 4 + 2);
                double tt = sum0 + x0;
                c0 += (fabs(sum0) >= fabs(x0)) ? (sum0 - tt) + x0 : (x0 - tt) + sum0;
                sum0 = tt;
                tt = sum1 + x1;
                c1 += (fabs(sum1) >= fabs(x1)) ? (sum1 - tt) + x1 : (x1 - tt) + sum1;
                sum1 = tt;
            }
            double* red = sRed;
            // warp butterfly on (sum, compensation) pairs, then warps in order
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double os = __shfl_xor_sync(0xffffffffu, sum0, o);
                const double oc = __shfl_xor_sync(0xffffffffu, c0, o);
                const double ps = __shfl_xor_sync(0xffffffffu, sum1, o);
                const double pc = __shfl_xor_sync(0xffffffffu, c1, o);
                const double ocnt = __shfl_xor_sync(0xffffffffu, cnt, o);
                double tt = sum0 + os;
                c0 += oc + ((fabs(sum0) >= fabs(os)) ? (sum0 - tt) + os : (os - tt) + sum0);
                sum0 = tt;
                tt = sum1 + ps;
                c1 += pc + ((fabs(sum1) >= fabs(ps)) ? (sum1 - tt) + ps : (ps - tt) + sum1);
                sum1 = tt;
                cnt += ocnt;
            }
            __syncthreads();
            if (lane == 0) {
                red[warp * 4 + 0] = sum0 + c0;
                red[warp * 4 + 1] = sum1 + c1;
                red[warp * 4 + 2] = cnt;
            }
            __syncthreads();
            if (tid == 0) {
                double S0 = 0, C0 = 0, S1 = 0, C1 = 0, N = 0;
                for (int w = 0; w < kWarps; ++w) {
                    double x = red[w * 4 + 0];
                    double tt = S0 + x;
                    C0 += (fabs(S0) >= fabs(x)) ? (S0 - tt) + x : (x - tt) + S0;
                    S0 = tt;
                    x = red[w * 4 + 1];
                    tt = S1 + x;
                    C1 += (fabs(S1) >= fabs(x)) ? (S1 - tt) + x : (x - tt) + S1;
                    S1 = tt;
                    N += red[w * 4 + 2];
                }
                if constexpr (OP == OP_ENERGY) {
                    p.out_scalar[0] = N > 0 ? __longlong_as_double(0x7ff0000000000000ll) : S0 + C0;
                    p.out_scalar[1] = S1 + C1;
                    p.out_scalar[2] = N;
                    p.out_scalar[3] = 0.0;
                } else if (p.out_scalar) {
                    p.out_scalar[0] = S0 + C0;
                }
                *p.tile_counter = 0u;
            }
        }
    }
    __syncthreads();
    if (tid == 0 && *sFlag) atomicOr(p.status, *sFlag);
}

}  // namespace fem
