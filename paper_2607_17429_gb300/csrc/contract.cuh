// Contraction of Eq. 15 for one flip and one right-hand side, specialised on the
// irrep dimension D so that no predicated work is issued for D < 5.
//
// rho tables are stored with padded rows: row length rho_row(D) elements (1, 2,
// 4, 4, 6 for D = 1..5, D rounded up to even above), so that an FP32 row is one
// 16-byte load (D = 3, 4) or 8-byte loads (D = 5; an 8-byte shared load with a
// few distinct addresses per warp takes one wavefront, a 16-byte load two), and
// an even-length row holds the element pairs of the packed FP32 FMA.
#pragma once

#include "common.cuh"

namespace ftlm {

__host__ __device__ constexpr int rho_row(int D) { return D == 1 ? 1 : (D == 3 ? 4 : D + (D & 1)); }

// elements of one padded table [G][D][rho_row(D)], rounded up to 16 bytes
template <typename VT>
__host__ __device__ inline int rho_table_elems(int G, int D) {
    const int n = G * D * rho_row(D);
    const int per16 = 16 / (int)sizeof(VT);
    return (n + per16 - 1) / per16 * per16;
}

template <typename VT, int RP>
__device__ __forceinline__ void load_row(const VT *p, VT (&r)[RP]) {
    if constexpr (sizeof(VT) == 4 && RP % 4 == 0) {
#pragma unroll
        for (int i = 0; i < RP / 4; ++i) {
            const float4 v = reinterpret_cast<const float4 *>(p)[i];
            r[4 * i] = v.x;
            r[4 * i + 1] = v.y;
            r[4 * i + 2] = v.z;
            r[4 * i + 3] = v.w;
        }
    } else if constexpr (sizeof(VT) == 4 && RP % 2 == 0) {
#pragma unroll
        for (int i = 0; i < RP / 2; ++i) {
            const float2 v = reinterpret_cast<const float2 *>(p)[i];
            r[2 * i] = v.x;
            r[2 * i + 1] = v.y;
        }
    } else if constexpr (sizeof(VT) == 8 && RP % 2 == 0) {
#pragma unroll
        for (int i = 0; i < RP / 2; ++i) {
            const double2 v = reinterpret_cast<const double2 *>(p)[i];
            r[2 * i] = v.x;
            r[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < RP; ++i) r[i] = p[i];
    }
}

// z[beta] += cf * sum_gamma rhoT(g)[beta][gamma] u[gamma], u = V_r' x_r' (x rows xr + k' B)
template <typename VT, int D>
__device__ __forceinline__ void contract_flip(const VT *__restrict__ R, const VT *__restrict__ xr, int B, int sid_j,
                                              int n_j, const VT *__restrict__ Vt, VT cf, VT *z) {
    constexpr int RP = rho_row(D);
    VT u[D];
    if (sid_j == 0) {
#pragma unroll
        for (int g2 = 0; g2 < D; ++g2) u[g2] = __ldg(xr + (size_t)g2 * B);
    } else {
#pragma unroll
        for (int g2 = 0; g2 < D; ++g2) u[g2] = (VT)0;
        for (int kp = 0; kp < n_j; ++kp) {
            const VT xv = __ldg(xr + (size_t)kp * B);
#pragma unroll
            for (int g2 = 0; g2 < D; ++g2) u[g2] += __ldg(Vt + g2 * D + kp) * xv;
        }
    }
#pragma unroll
    for (int be = 0; be < D; ++be) {
        VT row[RP];
        load_row<VT, RP>(R + be * RP, row);
        VT acc = row[0] * u[0];
#pragma unroll
        for (int ga = 1; ga < D; ++ga) acc += row[ga] * u[ga];
        z[be] += cf * acc;
    }
}

}  // namespace ftlm
