// Lees-Edwards boundary along z (Sec. 2.5: periodic in every direction with
// opposing velocities imposed on two parallel boundaries; cells crossing it
// continue on the other side).  The image above the box is displaced by
// D_n = U n (mod nx) in x and moves with U x^, the image below by -D_n, -U.
//
// Lattice: with the boundary on, collision and streaming use two arrays.
// le_collide_kernel collides every node in place of the other array (A ->
// B, natural order) and keeps the post-collision density and velocity of the
// two boundary planes; le_stream_kernel pulls the populations (B -> A): a
// population whose source lies across the plane is the linear interpolation
// in x, at the displaced position, of the two bracketing nodes of the
// opposite plane, each shifted by f_eq(rho*, u* +/- U) - f_eq(rho*, u*); it
// then writes the velocity with F/2 of the streamed populations.
//
// Coupling: vertices whose 4x4x4 stencil reaches across z = 0 or z = nz are
// kept in an extra bin (see bin_vertex).  For them each z-layer of the
// stencil that falls in an image uses the vertex's position displaced by
// -/+D_n in x (and, for interpolation, the image velocity +/-U x^):
// le_spread_kernel adds their forces into F with atomics after the bins'
// gather, le_interp_kernel interpolates and moves them.
#include "lattice_core.cuh"

namespace hemo {

namespace {

template <typename R>
__device__ __forceinline__ void peskin4_le(R t, R *w) {
    const R q = sqrt(R(1) + R(4) * t - R(4) * t * t);
    w[0] = (R(3) - R(2) * t - q) * R(0.125);
    w[1] = (R(3) - R(2) * t + q) * R(0.125);
    w[2] = (R(1) + R(2) * t + q) * R(0.125);
    w[3] = (R(1) + R(2) * t - q) * R(0.125);
}

// collision of every node, A (natural order) -> B (natural order)
template <typename T, typename R>
__global__ void __launch_bounds__(NODE_BX * NODE_BY) le_collide_kernel(View<R> v) {
    const int x = blockIdx.x * NODE_BX + threadIdx.x, y = blockIdx.y * NODE_BY + threadIdx.y, z = blockIdx.z;
    if (x >= v.nx || y >= v.ny) return;
    const size_t N = (size_t)v.N, n = (size_t)x + (size_t)v.nx * ((size_t)y + (size_t)v.ny * z);
    const T *A = (const T *)v.f;
    T *B = (T *)v.f2;
    R d[Q], p[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = Store<T>::ld(A[(size_t)i * N + n]);
    const R om = (v.ind && v.ind[n]) ? v.omega_in : v.omega;
    R rho, ux, uy, uz;
    bgk_guo<R>(d, v.F[n], v.F[N + n], v.F[2 * N + n], om, p, rho, ux, uy, uz);
#pragma unroll
    for (int i = 0; i < Q; ++i) B[(size_t)i * N + n] = Store<T>::st(p[i]);
    if (z == 0 || z == v.nz - 1) {  // post-collision moments of the stored values
        R s = R(0), mx = R(0), my = R(0), mz = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R q = Store<T>::ld(Store<T>::st(p[i]));
            s += q;
            if (cx(i)) mx += cx(i) > 0 ? q : -q;
            if (cy(i)) my += cy(i) > 0 ? q : -q;
            if (cz(i)) mz += cz(i) > 0 ? q : -q;
        }
        const R r = R(1) + s;
        R *o = v.le_aux + 4 * ((size_t)(z == 0 ? 0 : 1) * v.nx * v.ny + (size_t)y * v.nx + x);
        o[0] = r;
        o[1] = mx / r;
        o[2] = my / r;
        o[3] = mz / r;
    }
}

// f_eq_i(rho, u + dU x^) - f_eq_i(rho, u) with w = w_i
template <typename R>
__device__ __forceinline__ R eq_shift(int i, R w, R rho, R ux, R uy, R uz, R dU) {
    const R cu = R(cx(i)) * ux + R(cy(i)) * uy + R(cz(i)) * uz;
    const R cu2 = cu + R(cx(i)) * dU;
    const R uu = ux * ux + uy * uy + uz * uz, ux2 = ux + dU;
    const R uu2 = ux2 * ux2 + uy * uy + uz * uz;
    return w * rho * (R(3) * (cu2 - cu) + R(4.5) * (cu2 * cu2 - cu * cu) - R(1.5) * (uu2 - uu));
}

// pull streaming B -> A with the Lees-Edwards plane, then the velocity with
// F/2 of the streamed populations
template <typename T, typename R>
__global__ void __launch_bounds__(NODE_BX * NODE_BY) le_stream_kernel(View<R> v) {
    const int x = blockIdx.x * NODE_BX + threadIdx.x, y = blockIdx.y * NODE_BY + threadIdx.y, z = blockIdx.z;
    if (x >= v.nx || y >= v.ny) return;
    const size_t N = (size_t)v.N, n = (size_t)x + (size_t)v.nx * ((size_t)y + (size_t)v.ny * z);
    const T *B = (const T *)v.f2;
    T *A = (T *)v.f;
    const double D = le_shift(v);
    R d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int zs = z - cz(i), ys = wrap(y - cy(i), v.ny);
        if (zs >= 0 && zs < v.nz) {
            const int xs = wrap(x - cx(i), v.nx);
            d[i] = Store<T>::ld(B[(size_t)i * N + (size_t)xs + (size_t)v.nx * ((size_t)ys + (size_t)v.ny * zs)]);
        } else {
            const bool up = zs >= v.nz;  // from the image above (+D, +U) or below (-D, -U)
            const double xs = (double)(x - cx(i)) + (up ? -D : D);
            const double fl = floor(xs);
            const R wb = R(xs - fl);
            const int zb = up ? 0 : v.nz - 1;
            const R dU = R(up ? v.le_U : -v.le_U);
            R val = R(0);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int xk = wrap((int)fl + k, v.nx);
                const size_t sn = (size_t)xk + (size_t)v.nx * ((size_t)ys + (size_t)v.ny * zb);
                const R *a = v.le_aux + 4 * ((size_t)(up ? 0 : 1) * v.nx * v.ny + (size_t)ys * v.nx + xk);
                const R fk = Store<T>::ld(B[(size_t)i * N + sn]);
                val += (k ? wb : R(1) - wb) * (fk + eq_shift<R>(i, R(wgt(i)), a[0], a[1], a[2], a[3], dU));
            }
            d[i] = val;
        }
        A[(size_t)i * N + n] = Store<T>::st(d[i]);
    }
    R drho = R(0), mx = R(0), my = R(0), mz = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R q = Store<T>::ld(Store<T>::st(d[i]));
        drho += q;
        if (cx(i)) mx += cx(i) > 0 ? q : -q;
        if (cy(i)) my += cy(i) > 0 ? q : -q;
        if (cz(i)) mz += cz(i) > 0 ? q : -q;
    }
    const R inv = R(1) / (R(1) + drho);
    const R ux = (mx + R(0.5) * v.F[n]) * inv, uy = (my + R(0.5) * v.F[N + n]) * inv, uz = (mz + R(0.5) * v.F[2 * N + n]) * inv;
    v.u[n] = ux;
    v.u[N + n] = uy;
    v.u[2 * N + n] = uz;
    const float q = (float)(ux * ux + uy * uy + uz * uz);
    if (!(q < U_LIMIT2)) atomicOr(v.status, ST_NUMERIC);
}

// the layer c (-1..2 around the anchor) of a vertex's stencil: node z, x
// anchor and fraction, velocity offset of the image
template <typename R>
__device__ __forceinline__ void le_layer(const View<R> &v, double D, double X, int jz0, int c, int &zn, int &jx, R &tx,
                                        R &du) {
    int jz = jz0 + c;
    double xp = X;
    du = R(0);
    if (jz >= v.nz) {
        jz -= v.nz;
        xp = X - D;
        du = R(v.le_U);
    } else if (jz < 0) {
        jz += v.nz;
        xp = X + D;
        du = R(-v.le_U);
    }
    const double fl = floor(xp);
    zn = jz;
    jx = (int)fl;
    tx = R(xp - fl);
}

// forces of the vertices in the extra bin, 16 threads per vertex (one y-row
// b and z-layer c of the stencil each)
template <typename R>
__global__ void __launch_bounds__(256) le_spread_kernel(View<R> v) {
    const int s = v.start[v.nbins], e = v.start[v.nbins + 1];
    const int q = s + (blockIdx.x * blockDim.x + threadIdx.x) / 16;
    if (q >= e) return;
    const int r = threadIdx.x & 15, b = r & 3, c = r >> 2;
    const int i = v.perm[q];
    const double D = le_shift(v);
    const size_t N = (size_t)v.N;
    const int jx0 = v.anc_i[3 * (size_t)i], jy0 = v.anc_i[3 * (size_t)i + 1], jz0 = v.anc_i[3 * (size_t)i + 2];
    const R tx0 = v.anc_t[3 * (size_t)i], ty = v.anc_t[3 * (size_t)i + 1], tz = v.anc_t[3 * (size_t)i + 2];
    R wy[4], wz[4], wx[4];
    peskin4_le(ty, wy);
    peskin4_le(tz, wz);
    int zn, jx;
    R tx, du;
    le_layer(v, D, (double)jx0 + (double)tx0, jz0, c - 1, zn, jx, tx, du);
    peskin4_le(tx, wx);
    const int yn = wrap(jy0 - 1 + b, v.ny);
    const R wyz = wy[b] * wz[c];
    const R F0 = v.Fv[3 * (size_t)i], F1 = v.Fv[3 * (size_t)i + 1], F2 = v.Fv[3 * (size_t)i + 2];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int xn = wrap(jx - 1 + a, v.nx);
        const size_t n = (size_t)xn + (size_t)v.nx * ((size_t)yn + (size_t)v.ny * zn);
        const R w = wx[a] * wyz;
        atomicAdd(v.F + n, F0 * w);
        atomicAdd(v.F + N + n, F1 * w);
        atomicAdd(v.F + 2 * N + n, F2 * w);
    }
}

// interpolation and Euler move of the vertices in the extra bin, one
// thread per vertex
template <typename R>
__global__ void __launch_bounds__(256) le_interp_kernel(View<R> v) {
    const int s = v.start[v.nbins], e = v.start[v.nbins + 1];
    const int q = s + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= e) return;
    const int i = v.perm[q];
    const double D = le_shift(v);
    const size_t N = (size_t)v.N;
    const int jx0 = v.anc_i[3 * (size_t)i], jy0 = v.anc_i[3 * (size_t)i + 1], jz0 = v.anc_i[3 * (size_t)i + 2];
    const R tx0 = v.anc_t[3 * (size_t)i], ty = v.anc_t[3 * (size_t)i + 1], tz = v.anc_t[3 * (size_t)i + 2];
    R wy[4], wz[4];
    peskin4_le(ty, wy);
    peskin4_le(tz, wz);
    R U0 = R(0), U1 = R(0), U2 = R(0);
    for (int c = 0; c < 4; ++c) {
        int zn, jx;
        R tx, du, wx[4];
        le_layer(v, D, (double)jx0 + (double)tx0, jz0, c - 1, zn, jx, tx, du);
        peskin4_le(tx, wx);
        for (int b = 0; b < 4; ++b) {
            const int yn = wrap(jy0 - 1 + b, v.ny);
            const R wyz = wy[b] * wz[c];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int xn = wrap(jx - 1 + a, v.nx);
                const size_t n = (size_t)xn + (size_t)v.nx * ((size_t)yn + (size_t)v.ny * zn);
                const R w = wx[a] * wyz;
                U0 += w * (v.u[n] + du);
                U1 += w * v.u[N + n];
                U2 += w * v.u[2 * N + n];
            }
        }
    }
    R *o = v.off + 3 * (size_t)i;
    o[0] += U0;
    o[1] += U1;
    o[2] += U2;
}

__global__ void le_advance_kernel(long long *n) { *n += 1; }

}  // namespace

template <typename R>
void launch_le_lattice(const View<R> &v, int precision, cudaStream_t st) {
    const dim3 g((unsigned)((v.nx + NODE_BX - 1) / NODE_BX), (unsigned)((v.ny + NODE_BY - 1) / NODE_BY), (unsigned)v.nz),
        b(NODE_BX, NODE_BY);
    HEMO_DISPATCH_T(precision, R, (le_collide_kernel<T, R><<<g, b, 0, st>>>(v)));
    HEMO_DISPATCH_T(precision, R, (le_stream_kernel<T, R><<<g, b, 0, st>>>(v)));
}

template <typename R>
void launch_le_spread(const View<R> &v, cudaStream_t st) {
    // every vertex could be in the extra bin: the grid covers nv of them
    if (v.nv) le_spread_kernel<R><<<(unsigned)((16 * (size_t)v.nv + 255) / 256), 256, 0, st>>>(v);
}

template <typename R>
void launch_le_interp(const View<R> &v, cudaStream_t st) {
    if (v.nv) le_interp_kernel<R><<<(unsigned)((v.nv + 255) / 256), 256, 0, st>>>(v);
}

void launch_le_advance(long long *n, cudaStream_t st) { le_advance_kernel<<<1, 1, 0, st>>>(n); }

template void launch_le_lattice<double>(const View<double> &, int, cudaStream_t);
template void launch_le_lattice<float>(const View<float> &, int, cudaStream_t);
template void launch_le_spread<double>(const View<double> &, cudaStream_t);
template void launch_le_spread<float>(const View<float> &, cudaStream_t);
template void launch_le_interp<double>(const View<double> &, cudaStream_t);
template void launch_le_interp<float>(const View<float> &, cudaStream_t);

}  // namespace hemo
