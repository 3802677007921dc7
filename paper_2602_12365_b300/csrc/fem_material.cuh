// Compressible Neo-Hookean law on lane vectors (see fem_vec.cuh):
//   psi(F) = mu/2 (I1 - 3) - mu ln J + lam/2 (ln J)^2,  F = I + H,
//   P = dpsi/dF = mu (F - F^-T) + lam ln J F^-T,
//   dP = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T,
// (2D plane strain: F33 = 1 adds 1 to I1 and nothing else).
//
// FP32 accuracy: J - 1 is formed from the invariants of H (tr H, I2(H),
// det H) and F^-T - I from cof(I + H) = (1 + tr H) I - H^T + cof(H), so no
// quantity close to 1 is subtracted from 1; I1 - 3 = 2 tr H + H:H.
#pragma once
#include "fem_vec.cuh"

namespace fem {

template <int D, class V>
struct Kin {
    V G[D][D];  // F^-T - I
    V lnJ;
    V trH, HH;  // tr H, H:H
    int ok;     // bit c: component c has J > 0
};

template <int D, class V>
__device__ __forceinline__ void kinematics(const V (&H)[D][D], Kin<D, V>& k) {
    using S = typename VT<V>::S;
    const V one = splat<V>(S(1));
    k.trH = H[0][0];
#pragma unroll
    for (int i = 1; i < D; ++i) k.trH = k.trH + H[i][i];
    k.HH = H[0][0] * H[0][0];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j)
            if (i + j > 0) k.HH = vfma(H[i][j], H[i][j], k.HH);
    if constexpr (D == 2) {
        const V detH = vfma(H[0][0], H[1][1], -(H[0][1] * H[1][0]));
        const V Jm1 = k.trH + detH;
        const V J = one + Jm1;
        k.ok = vpos(J);
        const V rJ = vrcp(vsel(k.ok, J, S(1)));
        // cof(F) - J I = -det(H) I - H^T
        const V nrJ = -rJ;
        k.G[0][0] = (detH + H[0][0]) * nrJ;
        k.G[0][1] = H[1][0] * nrJ;
        k.G[1][0] = H[0][1] * nrJ;
        k.G[1][1] = (detH + H[1][1]) * nrJ;
        k.lnJ = vlog1p(vsel(k.ok, Jm1, S(0)));
    } else {
        V c[3][3];
        c[0][0] = vfma(H[1][1], H[2][2], -(H[1][2] * H[2][1]));
        c[0][1] = vfma(H[1][2], H[2][0], -(H[1][0] * H[2][2]));
        c[0][2] = vfma(H[1][0], H[2][1], -(H[1][1] * H[2][0]));
        c[1][0] = vfma(H[0][2], H[2][1], -(H[0][1] * H[2][2]));
        c[1][1] = vfma(H[0][0], H[2][2], -(H[0][2] * H[2][0]));
        c[1][2] = vfma(H[0][1], H[2][0], -(H[0][0] * H[2][1]));
        c[2][0] = vfma(H[0][1], H[1][2], -(H[0][2] * H[1][1]));
        c[2][1] = vfma(H[0][2], H[1][0], -(H[0][0] * H[1][2]));
        c[2][2] = vfma(H[0][0], H[1][1], -(H[0][1] * H[1][0]));
        const V I2 = c[0][0] + c[1][1] + c[2][2];
        const V detH = vfma(H[0][0], c[0][0], vfma(H[0][1], c[0][1], H[0][2] * c[0][2]));
        const V s = I2 + detH;
        const V Jm1 = k.trH + s;
        const V J = one + Jm1;
        k.ok = vpos(J);
        const V rJ = vrcp(vsel(k.ok, J, S(1)));
        // cof(F) - J I = cof(H) - H^T - (I2 + det H) I
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                V x = c[i][j] - H[j][i];
                if (i == j) x = x - s;
                k.G[i][j] = x * rJ;
            }
        k.lnJ = vlog1p(vsel(k.ok, Jm1, S(0)));
    }
}

// psi and the roundoff scale mu (I1/2 + |ln J|) + lam/2 ln^2 J
template <int D, class V>
__device__ __forceinline__ void density(const Kin<D, V>& k, V mu, V lam, V& psi, V& scale) {
    using S = typename VT<V>::S;
    const V half = splat<V>(S(0.5));
    const V l2 = half * lam * k.lnJ * k.lnJ;
    psi = vfma(mu, vfma(half, k.HH, k.trH - k.lnJ), l2);
    const V hI1 = vfma(half, k.HH, k.trH) + splat<V>(S(1.5));
    scale = vfma(mu, hI1 + vabs(k.lnJ), l2);
}

// P = mu (H - G) + lam lnJ (I + G)
template <int D, class V>
__device__ __forceinline__ void stress(const V (&H)[D][D], const Kin<D, V>& k, V mu, V lam,
                                       V (&P)[D][D]) {
    const V ll = lam * k.lnJ;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            V x = vfma(ll, k.G[i][j], mu * (H[i][j] - k.G[i][j]));
            if (i == j) x = x + ll;
            P[i][j] = x;
        }
}

// dP = mu dF + (mu - lam lnJ) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T
template <int D, class V>
__device__ __forceinline__ void tangent(const V (&dF)[D][D], const Kin<D, V>& k, V mu, V lam,
                                        V (&dP)[D][D]) {
    using S = typename VT<V>::S;
    const V one = splat<V>(S(1));
    V FiT[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) FiT[i][j] = (i == j) ? k.G[i][j] + one : k.G[i][j];
    V trA = FiT[0][0] * dF[0][0];  // tr(F^-1 dF) = F^-T : dF
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j)
            if (i + j > 0) trA = vfma(FiT[i][j], dF[i][j], trA);
    V M[D][D];  // dF^T F^-T
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            V s = dF[0][a] * FiT[0][j];
#pragma unroll
            for (int l = 1; l < D; ++l) s = vfma(dF[l][a], FiT[l][j], s);
            M[a][j] = s;
        }
    const V c1 = mu - lam * k.lnJ;
    const V c2 = lam * trA;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            V B = FiT[i][0] * M[0][j];
#pragma unroll
            for (int a = 1; a < D; ++a) B = vfma(FiT[i][a], M[a][j], B);
            dP[i][j] = vfma(c2, FiT[i][j], vfma(c1, B, mu * dF[i][j]));
        }
}

}  // namespace fem
