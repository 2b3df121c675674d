// Lattice kernels: fused D3Q19 BGK collision + streaming in place (AA
// pattern), post-streaming velocity, equilibrium initialisation, wall links
// and field read-out.
//
// Method: Sec. 2.2 (BGK update f_i(x + e_i, t + 1) = f_i + (f_i^eq - f_i) /
// tau, moments rho = sum f_i, u = sum f_i e_i / rho, second-order
// equilibrium, D3Q19, c_s^2 = 1/3), Sec. 2.3 (the membrane force enters as an
// external force term: Guo-Zheng-Shi source with the half-force velocity),
// Sec. 2.5 (no-slip walls by halfway bounce-back, moving walls, periodic
// edges).
//
// Storage: one array of 19*N deviations d_i = f_i - w_i (SoA, [i][n]),
// updated in place.  Even steps read and write the node's own 19 slots,
// writing the post-collision value of direction i into slot opp(i); odd steps
// read direction i from slot opp(i) of node x - c_i and write it into slot i
// of node x + c_i.  After an odd step the array is in natural order again.
// Bounce-back: a population whose target x + c_i is a wall is written back
// into slot opp(i) of its own node (odd step) or left in slot opp(i) with the
// moving-wall term applied (even step), where the next odd step reads it.
#include <type_traits>

#include "hemo_internal.cuh"

namespace hemo {

namespace {

// Read the 19 populations arriving at node n.  LAYOUT 0: natural order (slot
// i of n).  LAYOUT 1: after an even step (slot opp(i) of n - c_i, or slot i
// of n when n - c_i is a wall).
template <typename T, typename R, int LAYOUT>
__device__ __forceinline__ void load_pops(const View<R> &v, int n, uint64_t lk, const Nbr &o, R d[Q]) {
    const T *f = (const T *)v.f;
    const size_t N = (size_t)v.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (LAYOUT == 0) {
            d[i] = Store<T>::ld(f[(size_t)i * N + n]);
        } else {
            if (i == 0) {
                d[i] = Store<T>::ld(f[n]);
            } else if (link_code(lk, opp(i))) {
                d[i] = Store<T>::ld(f[(size_t)i * N + n]);
            } else {
                d[i] = Store<T>::ld(f[(size_t)opp(i) * N + n + o.of(-cx(i), -cy(i), -cz(i))]);
            }
        }
    }
}

template <typename T, typename R, int PARITY>
__global__ void __launch_bounds__(256) collide_stream_kernel(View<R> v) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) return;  // wall node
    const uint64_t lk = (nt & 0x80) ? v.links[n] : 0ull;
    const Nbr o = make_nbr(v, n);
    R d[Q];
    load_pops<T, R, PARITY>(v, n, lk, o, d);

    // moments of the deviations: rho = 1 + sum d, rho u = sum d c + F/2
    R rho = R(1), mx = R(0), my = R(0), mz = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += d[i];
        if (cx(i)) mx += cx(i) > 0 ? d[i] : -d[i];
        if (cy(i)) my += cy(i) > 0 ? d[i] : -d[i];
        if (cz(i)) mz += cz(i) > 0 ? d[i] : -d[i];
    }
    const size_t N = (size_t)v.N;
    const R Fx = v.F[n], Fy = v.F[N + n], Fz = v.F[2 * N + n];
    const R inv = R(1) / rho;
    const R ux = (mx + R(0.5) * Fx) * inv;
    const R uy = (my + R(0.5) * Fy) * inv;
    const R uz = (mz + R(0.5) * Fz) * inv;
    if (v.rec) {
        v.rec[n] = rho;
        v.rec[N + n] = ux;
        v.rec[2 * N + n] = uy;
        v.rec[3 * N + n] = uz;
    }
    const R uu = ux * ux + uy * uy + uz * uz;
    const R om = v.omega;
    const R src = R(1) - R(0.5) * om;
    const R uF = ux * Fx + uy * Fy + uz * Fz;

    T *f = (T *)v.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R w = R(wgt(i));
        const R cu = R(cx(i)) * ux + R(cy(i)) * uy + R(cz(i)) * uz;
        const R cF = R(cx(i)) * Fx + R(cy(i)) * Fy + R(cz(i)) * Fz;
        const R deq = w * ((rho - R(1)) + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));
        const R S = src * w * (R(3) * (cF - uF) + R(9) * cu * cF);
        R p = d[i] - om * (d[i] - deq) + S;
        const int code = link_code(lk, i);
        if (code) {
            const R cw = R(cx(i)) * v.uw[code][0] + R(cy(i)) * v.uw[code][1] + R(cz(i)) * v.uw[code][2];
            p -= R(6) * w * rho * cw;
        }
        if (PARITY == 0) {
            f[(size_t)opp(i) * N + n] = Store<T>::st(p);
        } else {
            if (code)
                f[(size_t)opp(i) * N + n] = Store<T>::st(p);
            else
                f[(size_t)i * N + n + o.of(cx(i), cy(i), cz(i))] = Store<T>::st(p);
        }
    }
}

// post-streaming velocity u = (sum f c + F/2) / rho with the force just
// applied; LAYOUT as in load_pops.  Flags non-finite or |u| > 0.3.
template <typename T, typename R, int LAYOUT>
__global__ void __launch_bounds__(256) moments_kernel(View<R> v) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) {
        if (v.rec) {  // recording into a fresh velocity buffer
            const int id = nt & 0x7f;
            v.u[n] = v.uw[id][0];
            v.u[(size_t)v.N + n] = v.uw[id][1];
            v.u[2 * (size_t)v.N + n] = v.uw[id][2];
        }
        return;
    }
    const uint64_t lk = (nt & 0x80) ? v.links[n] : 0ull;
    const Nbr o = make_nbr(v, n);
    R d[Q];
    load_pops<T, R, LAYOUT>(v, n, lk, o, d);
    R rho = R(1), mx = R(0), my = R(0), mz = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += d[i];
        if (cx(i)) mx += cx(i) > 0 ? d[i] : -d[i];
        if (cy(i)) my += cy(i) > 0 ? d[i] : -d[i];
        if (cz(i)) mz += cz(i) > 0 ? d[i] : -d[i];
    }
    const size_t N = (size_t)v.N;
    const R inv = R(1) / rho;
    const R ux = (mx + R(0.5) * v.F[n]) * inv;
    const R uy = (my + R(0.5) * v.F[N + n]) * inv;
    const R uz = (mz + R(0.5) * v.F[2 * N + n]) * inv;
    v.u[n] = ux;
    v.u[N + n] = uy;
    v.u[2 * N + n] = uz;
    const float q = (float)(ux * ux + uy * uy + uz * uz);
    if (!(q < U_LIMIT2)) atomicOr(v.status, ST_NUMERIC);
}

template <typename T, typename R>
__global__ void init_equilibrium_kernel(View<R> v, const double *u0) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    const size_t N = (size_t)v.N;
    T *f = (T *)v.f;
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) {
        const int id = nt & 0x7f;
        for (int i = 0; i < Q; ++i) f[(size_t)i * N + n] = Store<T>::st(R(0));
        v.u[n] = v.uw[id][0];
        v.u[N + n] = v.uw[id][1];
        v.u[2 * N + n] = v.uw[id][2];
        return;
    }
    double ux = 0, uy = 0, uz = 0;
    if (u0) {
        ux = u0[3 * (size_t)n];
        uy = u0[3 * (size_t)n + 1];
        uz = u0[3 * (size_t)n + 2];
    }
    const double uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        f[(size_t)i * N + n] = Store<T>::st(R(wgt(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu)));
    }
    v.u[n] = R(ux);
    v.u[N + n] = R(uy);
    v.u[2 * N + n] = R(uz);
}

template <typename T, typename R, int LAYOUT>
__global__ void populations_out_kernel(View<R> v, double *out) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    const uint8_t nt = v.ntype[n];
    double *o = out + (size_t)n * Q;
    if (nt & 0x7f) {
        for (int i = 0; i < Q; ++i) o[i] = wgt(i);
        return;
    }
    const uint64_t lk = (nt & 0x80) ? v.links[n] : 0ull;
    const Nbr nb = make_nbr(v, n);
    R d[Q];
    load_pops<T, R, LAYOUT>(v, n, lk, nb, d);
    for (int i = 0; i < Q; ++i) o[i] = wgt(i) + (double)d[i];
}

template <typename T, typename R, int LAYOUT>
__global__ void rho_out_kernel(View<R> v, R *out) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) {
        out[n] = R(0);
        return;
    }
    const uint64_t lk = (nt & 0x80) ? v.links[n] : 0ull;
    const Nbr nb = make_nbr(v, n);
    R d[Q];
    load_pops<T, R, LAYOUT>(v, n, lk, nb, d);
    R rho = R(1);
    for (int i = 0; i < Q; ++i) rho += d[i];
    out[n] = rho;
}

template <typename R>
__global__ void u_out_kernel(View<R> v, R *out) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    const size_t N = (size_t)v.N;
    out[3 * (size_t)n] = v.u[n];
    out[3 * (size_t)n + 1] = v.u[N + n];
    out[3 * (size_t)n + 2] = v.u[2 * N + n];
}

// Wall links: for each fluid node, the wall id of node + c_i (2 bits per
// direction; nodes beyond a non-periodic edge are resting walls).
__global__ void build_links_kernel(int nx, int ny, int nz, int px, int py, int pz, uint8_t *ntype,
                                   uint64_t *links) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nx * ny * nz) return;
    const uint8_t m = ntype[n];
    if (m) {  // wall node: keep its id, no links
        links[n] = 0;
        return;
    }
    const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    uint64_t lk = 0;
    for (int i = 1; i < Q; ++i) {
        int xx = x + cx(i), yy = y + cy(i), zz = z + cz(i);
        int code;
        if ((!px && (xx < 0 || xx >= nx)) || (!py && (yy < 0 || yy >= ny)) || (!pz && (zz < 0 || zz >= nz))) {
            code = 1;
        } else {
            xx = wrap(xx, nx);
            yy = wrap(yy, ny);
            zz = wrap(zz, nz);
            code = ntype[xx + nx * (yy + ny * zz)] & 0x7f;
        }
        lk |= (uint64_t)code << (2 * i);
    }
    links[n] = lk;
}

__global__ void mark_near_wall_kernel(int N, uint8_t *ntype, const uint64_t *links) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    if (ntype[n] == 0 && links[n] != 0) ntype[n] = 0x80;
}

// Natural-layout copy of the deviations (R, SoA [i][n]); wall nodes get 0.
template <typename T, typename R, int LAYOUT>
__global__ void copy_natural_kernel(View<R> v, R *out) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    const size_t N = (size_t)v.N;
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) {
        for (int i = 0; i < Q; ++i) out[(size_t)i * N + n] = R(0);
        return;
    }
    const uint64_t lk = (nt & 0x80) ? v.links[n] : 0ull;
    const Nbr o = make_nbr(v, n);
    R d[Q];
    load_pops<T, R, LAYOUT>(v, n, lk, o, d);
    for (int i = 0; i < Q; ++i) out[(size_t)i * N + n] = d[i];
}

// Inverse of copy_natural: writes natural-layout deviations into the
// in-place array in the layout of the given parity (0 natural; 1 the layout
// after an even step, where population i of node x sits in slot opp(i) of
// x - c_i, or in slot i of x when x - c_i is a wall).  Each slot is written
// by exactly one thread.
template <typename T, typename R, int LAYOUT>
__global__ void restore_natural_kernel(View<R> v, const R *in) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    const size_t N = (size_t)v.N;
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) return;
    T *f = (T *)v.f;
    const uint64_t lk = (nt & 0x80) ? v.links[n] : 0ull;
    const Nbr o = make_nbr(v, n);
    for (int i = 0; i < Q; ++i) {
        const T val = Store<T>::st(in[(size_t)i * N + n]);
        if (LAYOUT == 0 || i == 0) f[(size_t)i * N + n] = val;
        else if (link_code(lk, opp(i))) f[(size_t)i * N + n] = val;
        else f[(size_t)opp(i) * N + n + o.of(-cx(i), -cy(i), -cz(i))] = val;
    }
}

inline int nblocks(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
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

template <typename R>
void launch_collide(const View<R> &v, int precision, int parity, cudaStream_t st) {
    const int g = nblocks(v.N, 256);
    if (parity == 0)
        HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 0><<<g, 256, 0, st>>>(v)));
    else
        HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 1><<<g, 256, 0, st>>>(v)));
}

template <typename R>
void launch_moments(const View<R> &v, int precision, int parity, cudaStream_t st) {
    // after an even step the array is in the swapped layout (1), after an odd
    // step in natural order (0)
    const int g = nblocks(v.N, 256);
    if (parity == 0)
        HEMO_DISPATCH_T(precision, R, (moments_kernel<T, R, 1><<<g, 256, 0, st>>>(v)));
    else
        HEMO_DISPATCH_T(precision, R, (moments_kernel<T, R, 0><<<g, 256, 0, st>>>(v)));
}

template <typename R>
void launch_init_equilibrium(const View<R> &v, int precision, const double *u_dev, cudaStream_t st) {
    HEMO_DISPATCH_T(precision, R, (init_equilibrium_kernel<T, R><<<nblocks(v.N, 256), 256, 0, st>>>(v, u_dev)));
}

template <typename R>
void launch_populations_out(const View<R> &v, int precision, int layout, double *out, cudaStream_t st) {
    const int g = nblocks(v.N, 256);
    if (layout == 0)
        HEMO_DISPATCH_T(precision, R, (populations_out_kernel<T, R, 0><<<g, 256, 0, st>>>(v, out)));
    else
        HEMO_DISPATCH_T(precision, R, (populations_out_kernel<T, R, 1><<<g, 256, 0, st>>>(v, out)));
}

template <typename R>
void launch_rho_out(const View<R> &v, int precision, int layout, R *out, cudaStream_t st) {
    const int g = nblocks(v.N, 256);
    if (layout == 0)
        HEMO_DISPATCH_T(precision, R, (rho_out_kernel<T, R, 0><<<g, 256, 0, st>>>(v, out)));
    else
        HEMO_DISPATCH_T(precision, R, (rho_out_kernel<T, R, 1><<<g, 256, 0, st>>>(v, out)));
}

template <typename R>
void launch_u_out(const View<R> &v, R *out, cudaStream_t st) {
    u_out_kernel<R><<<nblocks(v.N, 256), 256, 0, st>>>(v, out);
}

void launch_build_links(int nx, int ny, int nz, const int *per, uint8_t *ntype, uint64_t *links, cudaStream_t st) {
    const long long N = (long long)nx * ny * nz;
    build_links_kernel<<<nblocks(N, 256), 256, 0, st>>>(nx, ny, nz, per[0], per[1], per[2], ntype, links);
    mark_near_wall_kernel<<<nblocks(N, 256), 256, 0, st>>>((int)N, ntype, links);
}

template <typename R>
void launch_copy_natural(const View<R> &v, int precision, int layout, R *out, cudaStream_t st) {
    const int g = nblocks(v.N, 256);
    if (layout == 0)
        HEMO_DISPATCH_T(precision, R, (copy_natural_kernel<T, R, 0><<<g, 256, 0, st>>>(v, out)));
    else
        HEMO_DISPATCH_T(precision, R, (copy_natural_kernel<T, R, 1><<<g, 256, 0, st>>>(v, out)));
}

template <typename R>
void launch_restore_natural(const View<R> &v, int precision, int layout, const R *in, cudaStream_t st) {
    const int g = nblocks(v.N, 256);
    if (layout == 0)
        HEMO_DISPATCH_T(precision, R, (restore_natural_kernel<T, R, 0><<<g, 256, 0, st>>>(v, in)));
    else
        HEMO_DISPATCH_T(precision, R, (restore_natural_kernel<T, R, 1><<<g, 256, 0, st>>>(v, in)));
}

#define HEMO_INST(R)                                                                              \
    template void launch_collide<R>(const View<R> &, int, int, cudaStream_t);                     \
    template void launch_moments<R>(const View<R> &, int, int, cudaStream_t);                     \
    template void launch_init_equilibrium<R>(const View<R> &, int, const double *, cudaStream_t); \
    template void launch_populations_out<R>(const View<R> &, int, int, double *, cudaStream_t);   \
    template void launch_rho_out<R>(const View<R> &, int, int, R *, cudaStream_t);                \
    template void launch_u_out<R>(const View<R> &, R *, cudaStream_t);                           \
    template void launch_copy_natural<R>(const View<R> &, int, int, R *, cudaStream_t);           \
    template void launch_restore_natural<R>(const View<R> &, int, int, const R *, cudaStream_t);
HEMO_INST(double)
HEMO_INST(float)

}  // namespace hemo
