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
    V Jm1;      // J - 1
    V trH, HH;  // tr H, H:H
    int ok;     // bit c: component c has J > 0
};

// BF: ln J by the branch-free FP32 logarithm (vlog1p_bf) instead of vlog1p
template <int D, class V, bool BF = false>
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
        k.Jm1 = Jm1;
        const V J = one + Jm1;
        k.ok = vpos(J);
        const V rJ = vrcp(vsel(k.ok, J, S(1)));
        // cof(F) - J I = -det(H) I - H^T
        const V nrJ = -rJ;
        k.G[0][0] = (detH + H[0][0]) * nrJ;
        k.G[0][1] = H[1][0] * nrJ;
        k.G[1][0] = H[0][1] * nrJ;
        k.G[1][1] = (detH + H[1][1]) * nrJ;
        if constexpr (BF)
            k.lnJ = vlog1p_bf(vsel(k.ok, Jm1, S(0)));
        else
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
        k.Jm1 = Jm1;
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
        if constexpr (BF)
            k.lnJ = vlog1p_bf(vsel(k.ok, Jm1, S(0)));
        else
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

// ---------------------------------------------------------------------------
// Neural constitutive model: psi = [NN(I1, J) - NN(3, 1)] + psi_NH.  The
// network enters through per-element coefficients evaluated at the element's
// (I1, J) and scaled here by w det J: C2 = psi_I1, C3 = psi_J, C11, C12, C22
// its second derivatives.  dpsi_NN/dF = 2 psi_I1 F + psi_J J F^-T.
// ---------------------------------------------------------------------------
template <int D, class V>
struct NcmCoef {
    V C2, C3, C11, C12, C22;
};

// P = mu (H - G) + lam lnJ (I + G) + 2 C2 (I + H) + C3 J (I + G)
template <int D, class V>
__device__ __forceinline__ void stress_ncm(const V (&H)[D][D], const Kin<D, V>& k, V mu, V lam,
                                           const NcmCoef<D, V>& c, V (&P)[D][D]) {
    using S = typename VT<V>::S;
    const V ll = lam * k.lnJ;
    const V cj = c.C3 * (splat<V>(S(1)) + k.Jm1);
    const V c2 = c.C2 + c.C2;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            V x = vfma(ll + cj, k.G[i][j], vfma(c2, H[i][j], mu * (H[i][j] - k.G[i][j])));
            if (i == j) x = x + ll + cj + c2;
            P[i][j] = x;
        }
}

// dP = mu dF + (mu - lam lnJ) B + lam trA F^-T                 (Neo-Hookean)
//    + 2 C2 dF + 2 (C11 dI1 + C12 dJ) F + J (C12 dI1 + C22 dJ) F^-T
//    + C3 (dJ F^-T - J B),
// B = F^-T dF^T F^-T, trA = tr(F^-1 dF), dJ = J trA, dI1 = 2 F : dF; the
// terms with B and F^-T share their tensors with the Neo-Hookean part.
template <int D, class V>
__device__ __forceinline__ void tangent_ncm(const V (&H)[D][D], const V (&dF)[D][D], const Kin<D, V>& k, V mu,
                                            V lam, const NcmCoef<D, V>& c, V (&dP)[D][D]) {
    using S = typename VT<V>::S;
    const V one = splat<V>(S(1));
    V FiT[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) FiT[i][j] = (i == j) ? k.G[i][j] + one : k.G[i][j];
    V trA = FiT[0][0] * dF[0][0];
    V FdF = dF[0][0];  // F : dF = tr dF + H : dF
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (i + j > 0) trA = vfma(FiT[i][j], dF[i][j], trA);
            if (i == j && i > 0) FdF = FdF + dF[i][j];
            FdF = vfma(H[i][j], dF[i][j], FdF);
        }
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
    const V J = one + k.Jm1;
    const V dJ = J * trA;
    const V dI1 = FdF + FdF;
    const V a2 = vfma(c.C11, dI1, c.C12 * dJ);
    const V fa = a2 + a2;                                              // coefficient of F
    const V cB = mu - vfma(lam, k.lnJ, c.C3 * J);                      // of B
    const V cF = vfma(lam, trA, vfma(J, vfma(c.C12, dI1, c.C22 * dJ), c.C3 * dJ));  // of F^-T
    const V cd = mu + c.C2 + c.C2;                                     // of dF
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            V B = FiT[i][0] * M[0][j];
#pragma unroll
            for (int a = 1; a < D; ++a) B = vfma(FiT[i][a], M[a][j], B);
            V x = vfma(cF, FiT[i][j], vfma(cB, B, vfma(fa, H[i][j], cd * dF[i][j])));
            if (i == j) x = x + fa;
            dP[i][j] = x;
        }
}

// NN part of a nodal diagonal block for the node gradient g, f = F g,
// q = F^-T g: 2 C2 |g|^2 I + 4 C11 f f^T + 2 C12 J (f q^T + q f^T) + C22 J^2 q q^T
// (the C3 terms cancel for dF = e_i g^T); added to the symmetric block in
// (00, 11, 22, 01, 02, 12) order (2D: 00, 11, 01)
template <int D, class V>
__device__ __forceinline__ void block_ncm(const V (&H)[D][D], const Kin<D, V>& k, const V (&g)[D], const V (&q)[D],
                                          const NcmCoef<D, V>& c, V (&out)[6]) {
    using S = typename VT<V>::S;
    V f[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        V s = g[i];
#pragma unroll
        for (int j = 0; j < D; ++j) s = vfma(H[i][j], g[j], s);
        f[i] = s;
    }
    const V J = splat<V>(S(1)) + k.Jm1;
    V n2 = g[0] * g[0];
#pragma unroll
    for (int i = 1; i < D; ++i) n2 = vfma(g[i], g[i], n2);
    const V d0 = (c.C2 + c.C2) * n2;
    const V a = splat<V>(S(4)) * c.C11, b = (c.C12 + c.C12) * J, e = c.C22 * J * J;
    auto ent = [&](int i, int j) { return vfma(a * f[i], f[j], vfma(b, vfma(f[i], q[j], q[i] * f[j]), e * q[i] * q[j])); };
    if constexpr (D == 3) {
        out[0] = out[0] + ent(0, 0) + d0;
        out[1] = out[1] + ent(1, 1) + d0;
        out[2] = out[2] + ent(2, 2) + d0;
        out[3] = out[3] + ent(0, 1);
        out[4] = out[4] + ent(0, 2);
        out[5] = out[5] + ent(1, 2);
    } else {
        out[0] = out[0] + ent(0, 0) + d0;
        out[1] = out[1] + ent(1, 1) + d0;
        out[2] = out[2] + ent(0, 1);
    }
}

}  // namespace fem
