// Collision arithmetic shared by the lattice kernels (AA in-place streaming
// and the two-array streaming of the Lees-Edwards boundary): the BGK update
// with the Guo source in pair form, and the dispatch over storage types.
#pragma once

#include <type_traits>

#include "hemo_internal.cuh"

namespace hemo {

// BGK collision with the Guo source at one node: from the 19 deviations d
// arriving at the node and the force F, the post-collision deviations p
// (before any wall term), the density and the velocity with F/2.
//
// Per direction, with d^eq = f^eq - w and S the Guo source,
//   p = (1 - om) d + om d^eq + S,
//   d^eq = w (rho - 1) + w rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u),
//   S = (1 - om/2) w (3 (c.F - u.F) + 9 (c.u)(c.F)).
// Directions come in opposite pairs (c, -c): the terms even in c are shared
// and the odd ones change sign, so each pair costs one c.u and one c.F.  In
// exact arithmetic the collision keeps the mass and adds F to the momentum;
// the rest population and the axis pairs' odd parts are computed so that
// rounded arithmetic keeps both too.
template <typename R>
__device__ __forceinline__ R recip(R x) {
    if constexpr (std::is_same<R, float>::value) return __frcp_rn(x);  // correctly rounded, as 1 / x
    else return R(1) / x;
}

template <typename R>
__device__ __forceinline__ void bgk_guo(const R (&d)[Q], R Fx, R Fy, R Fz, R om, R (&p)[Q], R &rho, R &ux, R &uy,
                                        R &uz) {
    // moments of the deviations: rho - 1 = sum d (summed without the 1, so
    // that FP32 keeps the density deviation's own precision), rho u = sum d c
    // + F/2
    R drho = R(0), mx = R(0), my = R(0), mz = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += d[i];
        if (cx(i)) mx += cx(i) > 0 ? d[i] : -d[i];
        if (cy(i)) my += cy(i) > 0 ? d[i] : -d[i];
        if (cz(i)) mz += cz(i) > 0 ? d[i] : -d[i];
    }
    rho = R(1) + drho;
    const R inv = recip(rho);
    ux = (mx + R(0.5) * Fx) * inv;
    uy = (my + R(0.5) * Fy) * inv;
    uz = (mz + R(0.5) * Fz) * inv;
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R om1 = R(1) - om, src = R(1) - R(0.5) * om;
    // even part A + (c.u) (B (c.u) + C (c.F)) of om d^eq + S and odd part
    // G (c.u) + H (c.F), for the axis weight 1/18; the diagonal weight 1/36
    // is exactly half of it
    const R w1 = R(1.0 / 18.0), ow = om * w1, sw = src * w1;
    const R A = ow * (drho - R(1.5) * rho * uu) - R(3) * sw * uF;
    const R B = R(4.5) * ow * rho, C = R(9) * sw, G = R(3) * ow * rho, H = R(3) * sw;
    // The weights' rounding (18 fl(1/18) = 1 + 7e-9 in FP32) would scale the
    // momentum by the same factor in every collision, a drift that adds up
    // over the steps.  The odd parts of the three axis pairs are therefore
    // the remainders that make the post-collision momentum m + F (what the
    // formulas give in exact arithmetic), and the rest population the
    // remainder that conserves mass.
    R sx = R(0), sy = R(0), sz = R(0), se = R(0), od[6];
#pragma unroll
    for (int a = 7; a < Q; a += 2) {  // diagonal pairs: even part now, odd part kept
        const R cu = R(cx(a)) * ux + R(cy(a)) * uy + R(cz(a)) * uz;
        const R cF = R(cx(a)) * Fx + R(cy(a)) * Fy + R(cz(a)) * Fz;
        const R even = R(0.5) * (A + cu * (B * cu + C * cF));
        const R odd = R(0.5) * (G * cu + H * cF);
        p[a] = om1 * d[a] + even;
        p[a + 1] = om1 * d[a + 1] + even;
        od[(a - 7) / 2] = odd;
        se += even;
        if (cx(a)) sx += cx(a) > 0 ? odd : -odd;
        if (cy(a)) sy += cy(a) > 0 ? odd : -odd;
        if (cz(a)) sz += cz(a) > 0 ? odd : -odd;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // axis pairs (1, 2), (3, 4), (5, 6)
        const int a = 1 + 2 * k;
        const R cu = k == 0 ? ux : (k == 1 ? uy : uz);
        const R cF = k == 0 ? Fx : (k == 1 ? Fy : Fz);
        const R mk = k == 0 ? mx : (k == 1 ? my : mz);
        const R sk = k == 0 ? sx : (k == 1 ? sy : sz);
        const R even = A + cu * (B * cu + C * cF);
        const R odd = R(0.5) * (om * mk + cF) - sk;  // sum over pairs of 2 c odd = om m + F
        se += even;
        p[a] = om1 * d[a] + even + odd;
        p[a + 1] = om1 * d[a + 1] + even - odd;
    }
    p[0] = om1 * d[0] + (om * drho - R(2) * se);  // sum over directions of om d^eq + S = om (rho - 1)
#pragma unroll
    for (int a = 7; a < Q; a += 2) {
        p[a] += od[(a - 7) / 2];
        p[a + 1] -= od[(a - 7) / 2];
    }
}


// storage type by precision: FP64 arithmetic only with FP64 storage
#define HEMO_DISPATCH_T(prec, R, CALL)                           \
    do {                                                         \
        if constexpr (std::is_same<R, double>::value) {          \
            using T = double;                                    \
            CALL;                                                \
        } else if ((prec) == HEMO_F32) {                         \
            using T = float;                                     \
            CALL;                                                \
        } else if ((prec) == HEMO_F16DEV) {                      \
            using T = __half;                                    \
            CALL;                                                \
        } else {                                                 \
            using T = __nv_bfloat16;                             \
            CALL;                                                \
        }                                                        \
    } while (0)

}  // namespace hemo
