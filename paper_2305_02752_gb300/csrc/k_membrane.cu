// Membrane mechanics, one CTA per cell (Sec. 2.3: F_total = F_link + F_bend
// + F_area + F_volume; vertices are Lagrangian points of a triangulated
// membrane).
//
// A CTA stages its cell's vertex offsets in shared memory, re-bases the cell
// (centroid += mean offset, offsets -= mean, so the FP32 offsets stay small
// while the FP64 centroid carries the position), sums area and volume over
// the triangles in FP64, and accumulates the four force terms per vertex in
// shared memory before one coalesced write.  The edge and triangle tables
// arrive in a processing order sorted on the host by smallest vertex id, so
// that the lanes of a warp load nearby shared-memory records; the FP64
// adjoint, which scatters with shared-memory atomics, walks them with a
// coprime stride instead (lanes on far-apart mesh parts).  Energies (forms documented in
// hemo.h):
//   link   K L0 [eps^2/2 - 1/2 ln(1 - eps^2/m^2)],   eps = (L - L0)/L0
//   bend   1/2 kb (theta - theta0)^2, theta = signed angle between the
//          outward normals of the two triangles of an edge
//   area   1/2 k_area ((A - A0)/A0)^2,  volume 1/2 k_volume ((V - V0)/V0)^2
// Forces are minus the energy gradients; the dihedral-angle gradient is the
// standard one (Bridson et al. 2003): the wing vertices move along their
// triangle normals with weight |e| / |n|^2, the edge vertices carry the
// lever-rule remainder.
#include <algorithm>
#include <type_traits>

#include "hemo_internal.cuh"

namespace hemo {

namespace {

template <typename R> struct V3 {
    R x, y, z;
};
template <typename R> __device__ __forceinline__ V3<R> ld3(const R *p) { return {p[0], p[1], p[2]}; }
template <typename R> __device__ __forceinline__ V3<R> operator-(V3<R> a, V3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename R> __device__ __forceinline__ V3<R> operator*(R s, V3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename R> __device__ __forceinline__ V3<R> operator+(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename R> __device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R> __device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R> __device__ __forceinline__ void sub_into(R *f, V3<R> a) {
    atomicAdd(f, -a.x);
    atomicAdd(f + 1, -a.y);
    atomicAdd(f + 2, -a.z);
}

__device__ __forceinline__ float sqrt_r(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqrt_r(double a) { return sqrt(a); }
__device__ __forceinline__ float atan2_r(float a, float b) { return atan2f(a, b); }
__device__ __forceinline__ double atan2_r(double a, double b) { return atan2(a, b); }
__device__ __forceinline__ float log_r(float a) { return logf(a); }
__device__ __forceinline__ double log_r(double a) { return log(a); }

// block-wide sum of K doubles; every thread receives the totals
template <int K>
__device__ void block_sum(double (&val)[K], double (*scratch)[32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) val[k] += __shfl_down_sync(0xffffffffu, val[k], o);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < K; ++k) scratch[k][wid] = val[k];
    __syncthreads();
    for (int k = 0; k < K; ++k) {
        double s = 0;
        for (int w = 0; w < nw; ++w) s += scratch[k][w];
        val[k] = s;
    }
    __syncthreads();
}

// eigenvalues of a symmetric 3x3 matrix, closed form (Smith 1961)
__device__ void sym3_eig(double a00, double a11, double a22, double a01, double a02, double a12, double &lmax,
                         double &lmin) {
    const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    const double q = (a00 + a11 + a22) / 3.0;
    const double p2 = (a00 - q) * (a00 - q) + (a11 - q) * (a11 - q) + (a22 - q) * (a22 - q) + 2.0 * p1;
    if (p2 <= 0.0) {
        lmax = lmin = q;
        return;
    }
    const double p = sqrt(p2 / 6.0);
    const double b00 = (a00 - q) / p, b11 = (a11 - q) / p, b22 = (a22 - q) / p;
    const double b01 = a01 / p, b02 = a02 / p, b12 = a12 / p;
    double r = 0.5 * (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02));
    r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
    const double phi = acos(r) / 3.0;
    lmax = q + 2.0 * p * cos(phi);
    lmin = q + 2.0 * p * cos(phi + 2.0943951023931954923);
}

// block totals of K accumulators, returned to every thread
template <typename R, int K>
__device__ void block_total(Acc<R> (&acc)[K], double (&out)[K], double (*scratch)[32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k].add_shfl(o);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < K; ++k) scratch[k][wid] = acc[k].value();
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0;
        for (int w = 0; w < nw; ++w) t += scratch[threadIdx.x][w];
        scratch[threadIdx.x][31] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = scratch[k][31];
}

// block-wide sum of K values of R, returned to every thread
template <typename R, int K>
__device__ void block_sum_r(R (&val)[K], R (*scratch)[32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) val[k] += __shfl_down_sync(0xffffffffu, val[k], o);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < K; ++k) scratch[k][wid] = val[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        R t = R(0);
        for (int w = 0; w < nw; ++w) t += scratch[k][w];
        val[k] = t;
    }
    __syncthreads();
}

// One CTA per cell.
// mode 0 (the step): re-base the offsets (centroid += mean offset), area and
//   volume, membrane forces F_v = -grad E into Fv, and each vertex's anchor
//   (floor and fraction of X per axis), bin key and bin count;
// mode 1: statistics only, no writes to the state: stats[6c..] = centroid,
//   area, volume, deformation index.
//
// Forces are gathered, not scattered: an edge pass leaves six coefficients
// per edge in shared memory (link: F on v0 = s (x1 - x0); bending: the
// wing vertices get cb |e| n/|n|^2 of their triangle, the edge vertices the
// lever-rule combinations of both), then each vertex sums the terms of the
// edges it ends, the edges it is a wing of and its triangles, one loop per
// kind over a per-mesh incidence table (so the lanes of a warp take the
// same branch).  No atomics, and the summation order is fixed: the forces
// are reproducible bit for bit.
// CTA shapes of the cell kernels: NT = 256 threads sized so that three FP32
// cells share an SM (registers and shared memory), or the largest CTA for
// a cell that has an SM to itself (512 threads in FP32; FP64's larger
// register footprint would spill at 512)
template <typename R> struct CellMax { static constexpr int T = sizeof(R) == 4 ? 512 : 256; };
template <typename R, int NT> struct CellMinBlocks { static constexpr int B = NT == 256 && sizeof(R) == 4 ? 3 : 1; };

// 4-wide records in shared memory (16-byte aligned for FP32: one 128-bit load)
template <typename R> struct Q4 {
    R x, y, z, w;
};
template <typename R> __device__ __forceinline__ Q4<R> ld4(const R *p) {
    if constexpr (sizeof(R) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        return {q.x, q.y, q.z, q.w};
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        return {a.x, a.y, b.x, b.y};
    }
}
template <typename R> __device__ __forceinline__ V3<R> xyz(Q4<R> q) { return {q.x, q.y, q.z}; }
template <typename R> __device__ __forceinline__ void st4(R *p, R x, R y, R z, R w) {
    if constexpr (sizeof(R) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(x, y, z, w);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(x, y);
        reinterpret_cast<double2 *>(p)[1] = make_double2(z, w);
    }
}

template <typename R, int NT>
__global__ void __launch_bounds__(NT, CellMinBlocks<R, NT>::B) cell_kernel(View<R> v, int mode, double *stats) {
    if (mode == 0 && v.adapt && !v.adapt[2]) return;  // adaptive separation: the forces are held on this step
    const int c = blockIdx.x;
    const MeshDev<R> m = v.meshes[v.cell_type[c]];
    const int first = v.cell_first[c];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);  // nv*4: offsets from the (new) centroid, padded
    R *tn = xs + 4 * v.max_nv;                  // nt*4: n / |n|^2 and |n|
    R *es = tn + 4 * v.max_nt;                  // ne*4 per-edge force coefficients
    R *tl = es + 4 * v.max_ne;                  // nt: 1/2 dE_local/dA_t (local area term, if on)
    __shared__ double scratch[6][32];
    __shared__ R rscratch[3][32];
    __shared__ double cnew[3];
    __shared__ R csplit[2][3];  // the new centroid as R hi + lo
    __shared__ R cav[2];        // area and volume coefficients

    // mean offset: any shift works, the centroid takes what the offsets lose.
    // A thread's first KC vertices stay in registers between the two loops.
    constexpr int KC = 4;
    R oc[KC][3];
    R mean[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
        const int i = threadIdx.x + kk * (int)blockDim.x;
        if (i < m.nv) {
            const R *o = v.off + 3 * (size_t)(first + i);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                oc[kk][k] = o[k];
                mean[k] += oc[kk][k];
            }
        }
    }
    for (int i = threadIdx.x + KC * (int)blockDim.x; i < m.nv; i += blockDim.x) {
        const R *o = v.off + 3 * (size_t)(first + i);
        mean[0] += o[0];
        mean[1] += o[1];
        mean[2] += o[2];
    }
    block_sum_r<R, 3>(mean, rscratch);
    for (int k = 0; k < 3; ++k) mean[k] /= R(m.nv);
    auto rebase = [&](int i, const R *o0) {
        R r[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] = o0[k] - mean[k];
        st4(xs + 4 * i, r[0], r[1], r[2], R(0));
        if (mode == 0) {
            R *o = v.off + 3 * (size_t)(first + i);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                o[k] = r[k];
                if (v.off_rec) v.off_rec[3 * (size_t)(first + i) + k] = r[k];
                if (v.off_eval) v.off_eval[3 * (size_t)(first + i) + k] = r[k];  // positions of this evaluation
            }
        }
    };
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
        const int i = threadIdx.x + kk * (int)blockDim.x;
        if (i < m.nv) rebase(i, oc[kk]);
    }
    for (int i = threadIdx.x + KC * (int)blockDim.x; i < m.nv; i += blockDim.x) {
        const R *o = v.off + 3 * (size_t)(first + i);
        const R ol[3] = {o[0], o[1], o[2]};
        rebase(i, ol);
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) cnew[k] = v.ctr[3 * c + k] + (double)mean[k];
        if (v.le && mode == 0) {  // Lees-Edwards: a centroid that left through z = 0 or nz moves to the other side
            const double D = le_shift(v);
            if (cnew[2] >= v.nz) {
                cnew[0] -= D;
                cnew[2] -= v.nz;
            } else if (cnew[2] < 0) {
                cnew[0] += D;
                cnew[2] += v.nz;
            }
        }
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) {
            csplit[0][k] = R(cnew[k]);
            csplit[1][k] = R(cnew[k] - (double)csplit[0][k]);
            if (mode == 0) {
                v.ctr[3 * c + k] = cnew[k];
                v.csp[6 * c + k] = csplit[0][k];
                v.csp[6 * c + 3 + k] = csplit[1][k];
            }
        }
    __syncthreads();

    if (mode == 0)  // anchors, keys and counts at the re-based positions
        for (int i = threadIdx.x; i < m.nv; i += blockDim.x)
            bin_vertex(v, (size_t)(first + i), csplit[0], csplit[1], xs + 4 * i);

    // per triangle: a = n / |n|^2 and |n|, with n = (x1 - x0) x (x2 - x0);
    // area |n|/2 and volume x0 . (x1 x x2) / 6 summed per cell
    // (the next item's mesh records are loaded before this item is
    // processed, here and in the edge pass: their L2 latency overlaps the
    // arithmetic)
    Acc<R> av[2];
    {
        int4 Tn = threadIdx.x < m.nt ? __ldg(m.tri4 + threadIdx.x) : make_int4(0, 0, 0, 0);
        for (int t = threadIdx.x; t < m.nt; t += blockDim.x) {
            const int4 T = Tn;
            if (t + (int)blockDim.x < m.nt) Tn = __ldg(m.tri4 + t + blockDim.x);
            if (!index_ok(T.x >= 0 && T.x < m.nv && T.y >= 0 && T.y < m.nv && T.z >= 0 && T.z < m.nv, v.status))
                continue;
            const V3<R> p0 = xyz(ld4(xs + 4 * T.x)), p1 = xyz(ld4(xs + 4 * T.y)), p2 = xyz(ld4(xs + 4 * T.z));
            const V3<R> n = cross(p1 - p0, p2 - p0);
            const R q = dot(n, n), ln = sqrt_r(q), iq = R(1) / q;
            st4(tn + 4 * t, iq * n.x, iq * n.y, iq * n.z, ln);
            if (m.k_local > R(0)) {
                const R a0 = __ldg(m.At0 + t);
                tl[t] = R(0.5) * m.k_local * (R(0.5) * ln - a0) / a0;
            }
            av[0].add(R(0.5) * ln);
            av[1].add(dot(p0, cross(p1, p2)) / R(6));
        }
    }
    double AV[2];
    block_total<R, 2>(av, AV, scratch);  // (synchronises: tn is complete below)
    const double A = AV[0], V = AV[1];

    if (mode == 1) {
        Acc<R> G[6];
        for (int i = threadIdx.x; i < m.nv; i += blockDim.x) {
            const R x = xs[4 * i], y = xs[4 * i + 1], z = xs[4 * i + 2];
            G[0].add(x * x);
            G[1].add(y * y);
            G[2].add(z * z);
            G[3].add(x * y);
            G[4].add(x * z);
            G[5].add(y * z);
        }
        double Gt[6];
        block_total<R, 6>(G, Gt, scratch);
        if (threadIdx.x == 0) {
            double lmax, lmin;
            const double in = 1.0 / m.nv;
            sym3_eig(Gt[0] * in, Gt[1] * in, Gt[2] * in, Gt[3] * in, Gt[4] * in, Gt[5] * in, lmax, lmin);
            const double a = sqrt(lmax), b = sqrt(lmin > 0 ? lmin : 0);
            double *o = stats + 6 * (size_t)c;
            o[0] = cnew[0];
            o[1] = cnew[1];
            o[2] = cnew[2];
            o[3] = A;
            o[4] = V;
            o[5] = (a - b) / (a + b);
        }
        return;
    }
    if (threadIdx.x == 0) {  // once per cell: FP64 is slow on this GPU
        cav[0] = R(0.5 * m.k_area * (A - m.A0) / (m.A0 * m.A0));
        cav[1] = R(m.k_volume * (V - m.V0) / (m.V0 * m.V0) / 6.0);
    }

    // per edge: link coefficient s (F on v0 = s (x1 - x0)), cb |e| for the
    // wing vertices, and the lever-rule coefficients cb sa0, cb sb0 of v0
    // (those of v1 are cb sa0 + cb |e| and cb sb0 + cb |e|, since
    // sa1 - sa0 = sb1 - sb0 = |e|); the edge's triangles are (v0, v1, a)
    // and (v1, v0, b)
    const int4 *edge4 = reinterpret_cast<const int4 *>(m.edge);  // v0, v1, a, b
    const int2 *etri2 = reinterpret_cast<const int2 *>(m.etri);
    int4 En = make_int4(0, 0, 0, 0);
    int2 Tn = make_int2(0, 0);
    R il0n = R(0), th0n = R(0);
    if (threadIdx.x < m.ne) {
        En = __ldg(edge4 + threadIdx.x);
        Tn = __ldg(etri2 + threadIdx.x);
        il0n = __ldg(m.invL0 + threadIdx.x);
        th0n = __ldg(m.th0 + threadIdx.x);
    }
    for (int e = threadIdx.x; e < m.ne; e += blockDim.x) {
        const int4 E = En;
        const int2 T = Tn;
        const R il0 = il0n, th0 = th0n;
        if (e + (int)blockDim.x < m.ne) {
            En = __ldg(edge4 + e + blockDim.x);
            Tn = __ldg(etri2 + e + blockDim.x);
            il0n = __ldg(m.invL0 + e + blockDim.x);
            th0n = __ldg(m.th0 + e + blockDim.x);
        }
        if (!index_ok(E.x >= 0 && E.x < m.nv && E.y >= 0 && E.y < m.nv && E.z >= 0 && E.z < m.nv && E.w >= 0 &&
                          E.w < m.nv && T.x >= 0 && T.x < m.nt && T.y >= 0 && T.y < m.nt,
                      v.status))
            continue;
        const V3<R> p0 = xyz(ld4(xs + 4 * E.x)), p1 = xyz(ld4(xs + 4 * E.y));
        const V3<R> pa = xyz(ld4(xs + 4 * E.z)), pb = xyz(ld4(xs + 4 * E.w));
        const V3<R> ed = p1 - p0;
        const R L = sqrt_r(dot(ed, ed));
        const R iL = R(1) / L;
        const R eps = L * il0 - R(1);
        const R den = m.m2 - eps * eps;
        if (!(den > R(0))) atomicOr(v.status, ST_NUMERIC);
        const R dEdL = m.K * (eps + eps / den);
        const V3<R> a1 = xyz(ld4(tn + 4 * T.x)), a2 = xyz(ld4(tn + 4 * T.y));  // n / |n|^2
        const R th = atan2_r(dot(cross(a1, a2), ed) * iL, dot(a1, a2));
        const R dth = th - th0;
        R cb = m.kb * dth;  // dE/dtheta
        if (m.thm2i > R(0)) {  // nonlinear bending
            const R r2 = dth * dth * m.thm2i;
            if (!(r2 < R(1))) atomicOr(v.status, ST_NUMERIC);
            cb = cb / (R(1) - r2);
        }
        st4(es + 4 * e, dEdL * iL, cb * L, cb * (dot(pa - p1, ed) * iL), cb * (dot(pb - p1, ed) * iL));
    }
    __syncthreads();

    // per vertex: the sum over its edges and triangles, walking the fan
    // T_k = (i, j_k, j_k+1) in cyclic order so that each triangle record and
    // each neighbour position is loaded once: at step k the edge (i, j_k)
    // (link and lever-rule bending; its triangles are T_k and T_k-1) and the
    // triangle T_k-1 (wing term of its edge opposite i, area and volume)
    const R ha = cav[0], sv = cav[1];
    for (int i = threadIdx.x; i < m.nv; i += blockDim.x) {
        const V3<R> pi = xyz(ld4(xs + 4 * i));
        V3<R> f = {R(0), R(0), R(0)};
        int4 g = __ldg(m.vfan + i);  // slot 0: the last entry
        int4 gn = __ldg(m.vfan + (size_t)m.nv + i);  // slot 1, requested ahead (its L2 latency overlaps slot 0's use)
        auto fan_ok = [&](int4 q) {
            return index_ok(q.x >= 0 && q.x < m.nt && q.y >= 0 && q.y < m.nv && (q.z >> 1) >= 0 && (q.z >> 1) < m.ne &&
                                q.w >= 0 && q.w < m.ne,
                            v.status);
        };
        if (!fan_ok(g)) continue;
        Q4<R> ap = ld4(tn + 4 * g.x);  // T_k-1: n / |n|^2 and |n|
        V3<R> xp = xyz(ld4(xs + 4 * g.y));  // position of j_k-1
        int op = g.w;  // edge of T_k-1 opposite i
        int tp = g.x;  // T_k-1
        for (int k = 1; k <= m.maxv; ++k) {
            g = gn;
            if (g.x < 0 || !fan_ok(g)) break;
            if (k < m.maxv) gn = __ldg(m.vfan + (size_t)(k + 1) * m.nv + i);  // the next slot, ahead
            const Q4<R> ak = ld4(tn + 4 * g.x);
            const V3<R> xk = xyz(ld4(xs + 4 * g.y));
            const Q4<R> cf = ld4(es + 4 * (g.z >> 1));
            // the edge's triangles (v0, v1, a), (v1, v0, b) are T_k, T_k-1
            // when i is its v0 (role 0) and T_k-1, T_k otherwise
            const bool r1 = g.z & 1;
            const V3<R> a1 = r1 ? xyz(ap) : xyz(ak), a2 = r1 ? xyz(ak) : xyz(ap);
            const V3<R> lk = cf.x * (xk - pi);
            f = r1 ? f + lk - ((cf.z + cf.y) * a1 + (cf.w + cf.y) * a2) : f + lk + (cf.z * a1 + cf.w * a2);
            f = f + es[4 * op + 1] * xyz(ap);
            const V3<R> nh = ap.w * xyz(ap);  // unit normal of T_k-1
            const R hk = m.k_local > R(0) ? ha + tl[tp] : ha;  // global and local area terms
            f = f - (hk * cross(nh, xk - xp) + sv * cross(xp, xk));
            ap = ak;
            xp = xk;
            op = g.w;
            tp = g.x;
        }
        R *o = v.Fv + 3 * (size_t)(first + i);
        o[0] = f.x;
        o[1] = f.y;
        o[2] = f.z;
    }
}

// ---------------------------------------------------------------------------
// Differentiation form
// ---------------------------------------------------------------------------
// Forward-mode dual number: value and derivative along one direction.
template <typename R> struct Dual {
    R v, t;
};
template <typename R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return {a.v + b.v, a.t + b.t}; }
template <typename R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return {a.v - b.v, a.t - b.t}; }
template <typename R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) {
    return {a.v * b.v, a.v * b.t + a.t * b.v};
}
template <typename R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, Dual<R> b) {
    return {a.v / b.v, (a.t * b.v - a.v * b.t) / (b.v * b.v)};
}
template <typename R> __device__ __forceinline__ Dual<R> dconst(R x) { return {x, R(0)}; }
template <typename R> __device__ __forceinline__ Dual<R> dsqrt(Dual<R> a) {
    const R s = sqrt_r(a.v);
    return {s, a.t / (R(2) * s)};
}
template <typename R> __device__ __forceinline__ Dual<R> datan2(Dual<R> y, Dual<R> x) {
    return {atan2_r(y.v, x.v), (x.v * y.t - y.v * x.t) / (x.v * x.v + y.v * y.v)};
}
template <typename R> __device__ __forceinline__ V3<Dual<R>> dld3(const R *pv, const R *pt) {
    return {{pv[0], pt[0]}, {pv[1], pt[1]}, {pv[2], pt[2]}};
}
template <typename R> __device__ __forceinline__ V3<R> vals(V3<Dual<R>> a) { return {a.x.v, a.y.v, a.z.v}; }
template <typename R> __device__ __forceinline__ V3<R> tans(V3<Dual<R>> a) { return {a.x.t, a.y.t, a.z.t}; }
template <typename R> __device__ __forceinline__ void add_into(R *f, R s, V3<R> a) {
    atomicAdd(f, s * a.x);
    atomicAdd(f + 1, s * a.y);
    atomicAdd(f + 2, s * a.z);
}

// Adjoint of the membrane forces of one cell (`slices` CTAs per cell: each
// computes the cell's triangle records, area and volume, then its share of
// the edge and triangle terms, and adds its part of the product to lamX,
// atomically when a cell has several CTAs), at the
// positions X_n left by the forward recomputation (cell_kernel mode 0):
//   lamX += (dF/dX) lamFv  -- F = -grad E, so dF/dX = -Hessian is symmetric
//                            and its product with lamFv is the derivative
//                            of F along lamFv, taken with dual numbers;
//   grad[4 type + k] += lamFv . F_k / modulus_k for the four terms (each is
//                            linear in its modulus).
template <typename R, int NT>
__global__ void __launch_bounds__(NT, CellMinBlocks<R, NT>::B) cell_adjoint_kernel(View<R> v, AdjView<R> a, int slices) {
    using D = Dual<R>;
    const int c = blockIdx.x / slices, slice = blockIdx.x % slices;
    const int type = v.cell_type[c];
    const MeshDev<R> m = v.meshes[type];
    const int first = v.cell_first[c];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);  // positions (relative to the centroid)
    R *xt = xs + 3 * v.max_nv;                  // direction: lamFv
    R *ft = xt + 3 * v.max_nv;                  // derivative of the forces along lamFv
    R *tn = ft + 3 * v.max_nv;                  // per triangle: n (3), dn (3), 1/|n|^2, its derivative
    __shared__ double scratch[6][32];
    for (int i = threadIdx.x; i < 3 * m.nv; i += blockDim.x) {  // re-based offsets of the forward step
        xs[i] = v.off[3 * (size_t)first + i];
        xt[i] = a.lamFv[3 * (size_t)first + i];
        ft[i] = R(0);
    }
    __syncthreads();

    Acc<R> av[4];  // A, dA, V, dV
    for (int t = threadIdx.x; t < m.nt; t += blockDim.x) {
        const int j0 = m.tri[3 * t], j1 = m.tri[3 * t + 1], j2 = m.tri[3 * t + 2];
        const V3<D> p0 = dld3(xs + 3 * j0, xt + 3 * j0), p1 = dld3(xs + 3 * j1, xt + 3 * j1),
                    p2 = dld3(xs + 3 * j2, xt + 3 * j2);
        const V3<D> n = cross(p1 - p0, p2 - p0);
        const D q = dot(n, n);
        const D iq = dconst(R(1)) / q;
        R *o = tn + 8 * t;
        o[0] = n.x.v; o[1] = n.y.v; o[2] = n.z.v;
        o[3] = n.x.t; o[4] = n.y.t; o[5] = n.z.t;
        o[6] = iq.v; o[7] = iq.t;
        const D ar = dconst(R(0.5)) * dsqrt(q);
        const D vo = dot(p0, cross(p1, p2));
        av[0].add(ar.v);
        av[1].add(ar.t);
        av[2].add(vo.v / R(6));
        av[3].add(vo.t / R(6));
    }
    double AV[4];
    block_total<R, 4>(av, AV, scratch);  // (synchronises: tn is complete below)
    __shared__ R cuv[4];  // the area and volume strain factors and their derivatives, FP64 once per cell
    if (threadIdx.x == 0) {
        cuv[0] = R((AV[0] - m.A0) / (m.A0 * m.A0));
        cuv[1] = R(AV[1] / (m.A0 * m.A0));
        cuv[2] = R((AV[2] - m.V0) / (m.V0 * m.V0));
        cuv[3] = R(AV[3] / (m.V0 * m.V0));
    }
    __syncthreads();
    const D ua = {cuv[0], cuv[1]}, uv = {cuv[2], cuv[3]};
    const R kA = R(m.k_area), kV = R(m.k_volume);

    Acc<R> th[4];  // lamFv . unit-modulus forces: link, bend, area, volume
    const int step = slices * (int)blockDim.x;  // this CTA's share of the edge and triangle terms
    for (int qe = slice * (int)blockDim.x + threadIdx.x; qe < m.ne; qe += step) {
        const int e = (int)(((long long)qe * m.estride) % m.ne);
        const int i0 = m.edge[4 * e], i1 = m.edge[4 * e + 1], ia = m.edge[4 * e + 2], ib = m.edge[4 * e + 3];
        const int t1 = m.etri[2 * e], t2 = m.etri[2 * e + 1];
        const V3<D> p0 = dld3(xs + 3 * i0, xt + 3 * i0), p1 = dld3(xs + 3 * i1, xt + 3 * i1);
        const V3<D> pa = dld3(xs + 3 * ia, xt + 3 * ia), pb = dld3(xs + 3 * ib, xt + 3 * ib);
        const V3<R> l0 = ld3(xt + 3 * i0), l1 = ld3(xt + 3 * i1), la = ld3(xt + 3 * ia), lb = ld3(xt + 3 * ib);
        const V3<D> ed = p1 - p0;
        const D L = dsqrt(dot(ed, ed));
        const D iL = dconst(R(1)) / L;
        const D eps = L * dconst(m.invL0[e]) - dconst(R(1));
        const D den = dconst(m.m2) - eps * eps;
        const D dEdL = dconst(m.Ku) * (eps + eps / den);
        const V3<D> u0 = (dEdL * iL) * ed;  // unit link force on v0; -u0 on v1
        add_into(ft + 3 * i0, m.k_link, tans(u0));
        add_into(ft + 3 * i1, -m.k_link, tans(u0));
        th[0].add(dot(l0, vals(u0)) - dot(l1, vals(u0)));

        const V3<D> n1 = dld3(tn + 8 * t1, tn + 8 * t1 + 3), n2 = dld3(tn + 8 * t2, tn + 8 * t2 + 3);
        const D iq1 = {tn[8 * t1 + 6], tn[8 * t1 + 7]}, iq2 = {tn[8 * t2 + 6], tn[8 * t2 + 7]};
        const V3<D> a1 = iq1 * n1, a2 = iq2 * n2;
        const D thd = datan2(dot(cross(n1, n2), ed) * iL, dot(n1, n2));
        const D cb = dconst(m.kbu) * (thd - dconst(m.th0[e]));
        const D sa0 = dot(pa - p1, ed) * iL, sb0 = dot(pb - p1, ed) * iL;
        const D sa1 = dot(pa - p0, ed) * iL, sb1 = dot(pb - p0, ed) * iL;
        const V3<D> fa = (cb * L) * a1, fb = (cb * L) * a2;
        const V3<D> f0 = cb * (sa0 * a1 + sb0 * a2);
        const V3<D> f1 = (dconst(R(0)) - cb) * (sa1 * a1 + sb1 * a2);
        add_into(ft + 3 * ia, m.k_bend, tans(fa));
        add_into(ft + 3 * ib, m.k_bend, tans(fb));
        add_into(ft + 3 * i0, m.k_bend, tans(f0));
        add_into(ft + 3 * i1, m.k_bend, tans(f1));
        th[1].add(dot(la, vals(fa)) + dot(lb, vals(fb)) + dot(l0, vals(f0)) + dot(l1, vals(f1)));
    }
    for (int qt = slice * (int)blockDim.x + threadIdx.x; qt < m.nt; qt += step) {
        const int t = (int)(((long long)qt * m.tstride) % m.nt);
        const int j[3] = {m.tri[3 * t], m.tri[3 * t + 1], m.tri[3 * t + 2]};
        const V3<D> p[3] = {dld3(xs + 3 * j[0], xt + 3 * j[0]), dld3(xs + 3 * j[1], xt + 3 * j[1]),
                            dld3(xs + 3 * j[2], xt + 3 * j[2])};
        const D iq = {tn[8 * t + 6], tn[8 * t + 7]};
        const V3<D> nh = dsqrt(iq) * dld3(tn + 8 * t, tn + 8 * t + 3);
        for (int k = 0; k < 3; ++k) {
            const V3<D> &pk1 = p[(k + 1) % 3], &pk2 = p[(k + 2) % 3];
            const V3<D> fa = (dconst(R(-0.5)) * ua) * cross(nh, pk2 - pk1);
            const V3<D> fv = (dconst(R(-1) / R(6)) * uv) * cross(pk1, pk2);
            add_into(ft + 3 * j[k], kA, tans(fa));
            add_into(ft + 3 * j[k], kV, tans(fv));
            const V3<R> lk = ld3(xt + 3 * j[k]);
            th[2].add(dot(lk, vals(fa)));
            th[3].add(dot(lk, vals(fv)));
        }
    }
    double TH[4];
    block_total<R, 4>(th, TH, scratch);
    if (threadIdx.x < 4) atomicAdd(a.grad + 4 * type + threadIdx.x, TH[threadIdx.x]);
    __syncthreads();
    if (slices == 1)
        for (int i = threadIdx.x; i < 3 * m.nv; i += blockDim.x) a.lamX[3 * (size_t)first + i] += ft[i];
    else
        for (int i = threadIdx.x; i < 3 * m.nv; i += blockDim.x) atomicAdd(a.lamX + 3 * (size_t)first + i, ft[i]);
}

// FP32 form of the membrane adjoint as a gather, in the forward kernel's
// order: the triangle pass and the edge pass leave their records (as in
// cell_kernel) with their derivatives along lamFv, then each vertex walks
// its fan and sums its link, bending, area and volume terms as dual numbers.
// The derivative parts give the Hessian product (times the moduli) added to
// lamX; the value parts, dotted with lamFv, give the unit-modulus terms
// summed into the gradients of the four moduli.  No shared atomics.
//
// With fewer cells than SMs each cell takes `slices` CTAs: every CTA builds
// the cell's triangle and edge records, then walks the fans of its share of
// the vertices only (each vertex's lamX written by one CTA; the modulus
// terms added with one atomic per CTA).
template <int NT>
__global__ void __launch_bounds__(NT, 1) cell_adjoint_gather_kernel(View<float> v, AdjView<float> a, int slices) {
    using R = float;
    using D = Dual<R>;
    const int c = blockIdx.x / slices, slice = blockIdx.x % slices;
    const int type = v.cell_type[c];
    const MeshDev<R> m = v.meshes[type];
    const int first = v.cell_first[c];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *xv = reinterpret_cast<R *>(smem_raw);  // nv*4 positions (relative to the centroid)
    R *xd = xv + 4 * v.max_nv;                 // nv*4 the direction lamFv
    R *tv = xd + 4 * v.max_nv;                 // nt*4 n / |n|^2 and |n|
    R *td = tv + 4 * v.max_nt;                 // nt*4 their derivatives
    R *ev = td + 4 * v.max_nt;                 // ne*4 edge coefficients (unit moduli)
    R *et = ev + 4 * v.max_ne;                 // ne*4 their derivatives
    __shared__ double scratch[6][32];
    __shared__ R cuv[4];  // unit-modulus area and volume factors and their derivatives
    auto dq = [](const R *pv, const R *pt) -> V3<D> {
        const float4 p = *reinterpret_cast<const float4 *>(pv), q = *reinterpret_cast<const float4 *>(pt);
        return {{p.x, q.x}, {p.y, q.y}, {p.z, q.z}};
    };
    auto st4 = [](R *o, R x, R y, R z, R w) { *reinterpret_cast<float4 *>(o) = make_float4(x, y, z, w); };
    for (int i = threadIdx.x; i < m.nv; i += blockDim.x) {  // re-based offsets of the forward step
        const R *o = v.off + 3 * (size_t)(first + i), *l = a.lamFv + 3 * (size_t)(first + i);
        st4(xv + 4 * i, o[0], o[1], o[2], R(0));
        st4(xd + 4 * i, l[0], l[1], l[2], R(0));
    }
    __syncthreads();

    Acc<R> av[4];  // A, dA, V, dV
    for (int t = threadIdx.x; t < m.nt; t += blockDim.x) {
        const int4 T = __ldg(m.tri4 + t);
        const V3<D> p0 = dq(xv + 4 * T.x, xd + 4 * T.x), p1 = dq(xv + 4 * T.y, xd + 4 * T.y),
                    p2 = dq(xv + 4 * T.z, xd + 4 * T.z);
        const V3<D> n = cross(p1 - p0, p2 - p0);
        const D q = dot(n, n), ln = dsqrt(q), iq = dconst(R(1)) / q;
        const V3<D> an = iq * n;
        st4(tv + 4 * t, an.x.v, an.y.v, an.z.v, ln.v);
        st4(td + 4 * t, an.x.t, an.y.t, an.z.t, ln.t);
        const D vo = dot(p0, cross(p1, p2));
        av[0].add(R(0.5) * ln.v);
        av[1].add(R(0.5) * ln.t);
        av[2].add(vo.v / R(6));
        av[3].add(vo.t / R(6));
    }
    double AV[4];
    block_total<R, 4>(av, AV, scratch);  // (synchronises: the triangle records are complete below)
    if (threadIdx.x == 0) {  // once per cell in FP64
        cuv[0] = R(0.5 * (AV[0] - m.A0) / (m.A0 * m.A0));
        cuv[1] = R(0.5 * AV[1] / (m.A0 * m.A0));
        cuv[2] = R((AV[2] - m.V0) / (m.V0 * m.V0) / 6.0);
        cuv[3] = R(AV[3] / (m.V0 * m.V0) / 6.0);
    }

    // per edge, unit moduli: link s (F on v0 = s (x1 - x0)), cb |e|, cb sa0, cb sb0
    for (int e = threadIdx.x; e < m.ne; e += blockDim.x) {
        const int4 E = __ldg(reinterpret_cast<const int4 *>(m.edge) + e);  // v0, v1, a, b
        const int2 T = __ldg(reinterpret_cast<const int2 *>(m.etri) + e);
        const V3<D> p0 = dq(xv + 4 * E.x, xd + 4 * E.x), p1 = dq(xv + 4 * E.y, xd + 4 * E.y);
        const V3<D> pa = dq(xv + 4 * E.z, xd + 4 * E.z), pb = dq(xv + 4 * E.w, xd + 4 * E.w);
        const V3<D> ed = p1 - p0;
        const D L = dsqrt(dot(ed, ed)), iL = dconst(R(1)) / L;
        const D eps = L * dconst(__ldg(m.invL0 + e)) - dconst(R(1));
        const D den = dconst(m.m2) - eps * eps;
        const D sl = dconst(m.Ku) * (eps + eps / den) * iL;
        const V3<D> a1 = dq(tv + 4 * T.x, td + 4 * T.x), a2 = dq(tv + 4 * T.y, td + 4 * T.y);
        const D th = datan2(dot(cross(a1, a2), ed) * iL, dot(a1, a2));
        const D cb = dconst(m.kbu) * (th - dconst(__ldg(m.th0 + e)));
        const D c1 = cb * L, c2 = cb * (dot(pa - p1, ed) * iL), c3 = cb * (dot(pb - p1, ed) * iL);
        st4(ev + 4 * e, sl.v, c1.v, c2.v, c3.v);
        st4(et + 4 * e, sl.t, c1.t, c2.t, c3.t);
    }
    __syncthreads();

    const D ha = {cuv[0], cuv[1]}, sv = {cuv[2], cuv[3]};
    const R kl = m.k_link, kb = m.k_bend, kA = R(m.k_area), kV = R(m.k_volume);
    Acc<R> th[4];  // lamFv . unit-modulus forces: link, bend, area, volume
    const int per = (m.nv + slices - 1) / slices, i0 = slice * per, i1 = min(m.nv, i0 + per);
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const V3<D> pi = dq(xv + 4 * i, xd + 4 * i);
        const V3<D> z = {dconst(R(0)), dconst(R(0)), dconst(R(0))};
        V3<D> fl = z, fb = z, fa = z, fv = z;
        int4 g = __ldg(m.vfan + i);  // slot 0: the last fan entry
        V3<D> ap = dq(tv + 4 * g.x, td + 4 * g.x);
        D aw = {tv[4 * g.x + 3], td[4 * g.x + 3]};
        V3<D> xp = dq(xv + 4 * g.y, xd + 4 * g.y);
        int op = g.w;
        for (int k = 1; k <= m.maxv; ++k) {
            g = __ldg(m.vfan + (size_t)k * m.nv + i);
            if (g.x < 0) break;
            const V3<D> ak = dq(tv + 4 * g.x, td + 4 * g.x);
            const D kw = {tv[4 * g.x + 3], td[4 * g.x + 3]};
            const V3<D> xk = dq(xv + 4 * g.y, xd + 4 * g.y);
            const int id = g.z >> 1;
            const float4 cv = *reinterpret_cast<const float4 *>(ev + 4 * id), ct = *reinterpret_cast<const float4 *>(et + 4 * id);
            const D cs = {cv.x, ct.x}, cl = {cv.y, ct.y}, ca = {cv.z, ct.z}, cbb = {cv.w, ct.w};
            const bool r1 = g.z & 1;
            const V3<D> a1 = r1 ? ap : ak, a2 = r1 ? ak : ap;
            fl = fl + cs * (xk - pi);
            fb = r1 ? fb - ((ca + cl) * a1 + (cbb + cl) * a2) : fb + (ca * a1 + cbb * a2);
            fb = fb + D{ev[4 * op + 1], et[4 * op + 1]} * ap;  // wing term of T_k-1's edge opposite i
            const V3<D> nh = aw * ap;                          // unit normal of T_k-1
            fa = fa - ha * cross(nh, xk - xp);
            fv = fv - sv * cross(xp, xk);
            ap = ak;
            aw = kw;
            xp = xk;
            op = g.w;
        }
        const V3<R> tl = tans(fl), tb = tans(fb), ta = tans(fa), tw = tans(fv);
        R *o = a.lamX + 3 * (size_t)(first + i);
        o[0] += kl * tl.x + kb * tb.x + kA * ta.x + kV * tw.x;
        o[1] += kl * tl.y + kb * tb.y + kA * ta.y + kV * tw.y;
        o[2] += kl * tl.z + kb * tb.z + kA * ta.z + kV * tw.z;
        const V3<R> lam = tans(pi);  // lamFv at this vertex
        th[0].add(dot(lam, vals(fl)));
        th[1].add(dot(lam, vals(fb)));
        th[2].add(dot(lam, vals(fa)));
        th[3].add(dot(lam, vals(fv)));
    }
    double TH[4];
    block_total<R, 4>(th, TH, scratch);
    if (threadIdx.x < 4) atomicAdd(a.grad + 4 * type + threadIdx.x, TH[threadIdx.x]);
}

// eigenvector of the symmetric 3x3 matrix g (xx, yy, zz, xy, xz, yz) for
// the eigenvalue lam: the longest cross product of two rows of g - lam I
__device__ void sym3_vec(const double *g, double lam, double *e) {
    const double r[3][3] = {{g[0] - lam, g[3], g[4]}, {g[3], g[1] - lam, g[5]}, {g[4], g[5], g[2] - lam}};
    double best = -1.0;
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b) {
            const double c[3] = {r[a][1] * r[b][2] - r[a][2] * r[b][1], r[a][2] * r[b][0] - r[a][0] * r[b][2],
                                 r[a][0] * r[b][1] - r[a][1] * r[b][0]};
            const double n2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
            if (n2 > best) {
                best = n2;
                const double s = n2 > 0 ? 1.0 / sqrt(n2) : 0.0;
                e[0] = c[0] * s;
                e[1] = c[1] * s;
                e[2] = c[2] * s;
            }
        }
}

// Deformation loss of each cell, DI + |centroid - c0|^2, with
// DI = (sqrt(l1) - sqrt(l3)) / (sqrt(l1) + sqrt(l3)) from the gyration tensor
// G = mean (X - c)(X - c)^T, and its gradient divided by the number of cells
// (the loss is the mean over cells): d l_k / dX_v = (2/n)(e_k . r_v) e_k.
template <typename R>
__global__ void __launch_bounds__(256) deformation_loss_kernel(View<R> v, const double *c0, double *cell_loss, R *dLdX) {
    const int c = blockIdx.x;
    const MeshDev<R> m = v.meshes[v.cell_type[c]];
    const int first = v.cell_first[c];
    __shared__ double scratch[6][32];
    __shared__ double coef[9];  // k1, k3, e1 (3), e3 (3), unused
    double mean[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < m.nv; i += blockDim.x)
        for (int k = 0; k < 3; ++k) mean[k] += (double)v.off[3 * (size_t)(first + i) + k];
    block_sum<3>(mean, scratch);
    for (int k = 0; k < 3; ++k) mean[k] /= m.nv;
    double G[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < m.nv; i += blockDim.x) {
        const double x = (double)v.off[3 * (size_t)(first + i)] - mean[0];
        const double y = (double)v.off[3 * (size_t)(first + i) + 1] - mean[1];
        const double z = (double)v.off[3 * (size_t)(first + i) + 2] - mean[2];
        G[0] += x * x; G[1] += y * y; G[2] += z * z;
        G[3] += x * y; G[4] += x * z; G[5] += y * z;
    }
    block_sum<6>(G, scratch);
    for (int k = 0; k < 6; ++k) G[k] /= m.nv;
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = v.ctr[3 * c + k] + mean[k] - c0[3 * c + k];
    if (threadIdx.x == 0) {
        double l1, l3;
        sym3_eig(G[0], G[1], G[2], G[3], G[4], G[5], l1, l3);
        const double aa = sqrt(l1), bb = sqrt(l3 > 0 ? l3 : 0);
        const double DI = (aa - bb) / (aa + bb);
        cell_loss[c] = DI + d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double k1 = 0, k3 = 0;
        if (aa - bb > 1e-12 * aa && bb > 0) {  // DI is not differentiable at isotropy
            k1 = 2.0 / m.nv * bb / (aa * (aa + bb) * (aa + bb));
            k3 = -2.0 / m.nv * aa / (bb * (aa + bb) * (aa + bb));
        }
        coef[0] = k1;
        coef[1] = k3;
        sym3_vec(G, l1, coef + 2);
        sym3_vec(G, l3, coef + 5);
    }
    __syncthreads();
    const double inv_nc = 1.0 / v.ncell;
    for (int i = threadIdx.x; i < m.nv; i += blockDim.x) {
        double r[3];
        for (int k = 0; k < 3; ++k) r[k] = (double)v.off[3 * (size_t)(first + i) + k] - mean[k];
        const double p1 = r[0] * coef[2] + r[1] * coef[3] + r[2] * coef[4];
        const double p3 = r[0] * coef[5] + r[1] * coef[6] + r[2] * coef[7];
        for (int k = 0; k < 3; ++k)
            dLdX[3 * (size_t)(first + i) + k] =
                R(inv_nc * (coef[0] * p1 * coef[2 + k] + coef[1] * p3 * coef[5 + k] + 2.0 * d[k] / m.nv));
    }
}

}  // namespace

// with no more cells than multiprocessors each cell has an SM to itself and
// the larger CTA shortens its latency; with more cells, 256 threads let
// three cells share an SM
template <typename R>
bool cell_wide(const View<R> &v) { return CellMax<R>::T > 256 && v.ncell <= v.nsm; }

template <typename R>
void launch_cell_forces(const View<R> &v, int mode, double *stats, cudaStream_t st) {
    if (v.ncell == 0) return;
    // positions and force accumulators of the largest mesh type
    const size_t smem = cell_smem_bytes<R>(v.max_nv, v.max_nt, v.max_ne);
    if (cell_wide(v)) cell_kernel<R, CellMax<R>::T><<<v.ncell, CellMax<R>::T, smem, st>>>(v, mode, stats);
    else cell_kernel<R, 256><<<v.ncell, 256, smem, st>>>(v, mode, stats);
}

template <typename R>
cudaError_t set_cell_smem_limit(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(cell_kernel<R, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && CellMax<R>::T != 256)
        e = cudaFuncSetAttribute(cell_kernel<R, CellMax<R>::T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

// CTAs per cell of the FP32 adjoint gather when cells are fewer than SMs
// (measured on the 48^3 box with 4 cells: reverse step 124.4 -> 119.7 us;
// 16 CTAs no better)
constexpr int ADJ_GATHER_SLICES = 8;
template <typename R>
void launch_cell_adjoint(const View<R> &v, const AdjView<R> &a, cudaStream_t st) {
    if (v.ncell == 0) return;
    if constexpr (std::is_same<R, float>::value) {
        const size_t gs = cell_adjoint_gather_bytes(v.max_nv, v.max_nt, v.max_ne);
        if (gs <= CELL_ADJ_GATHER_MAX_SMEM) {
            // few cells: several CTAs per cell, each gathering a share of
            // the vertices (the records are rebuilt by each)
            const int slices = std::max(1, std::min(ADJ_GATHER_SLICES, v.nsm / v.ncell));
            if (cell_wide(v))
                cell_adjoint_gather_kernel<CellMax<R>::T><<<v.ncell * slices, CellMax<R>::T, gs, st>>>(v, a, slices);
            else
                cell_adjoint_gather_kernel<256><<<v.ncell * slices, 256, gs, st>>>(v, a, slices);
            return;
        }
    }
    const size_t smem = cell_adjoint_smem_bytes<R>(v.max_nv, v.max_nt);
    // few cells: spread each over several CTAs (FP64 arithmetic is slow per
    // SM, so the work goes to as many SMs as there are)
    const int slices = std::max(1, std::min(32, v.nsm / v.ncell));
    if (slices == 1 && cell_wide(v)) cell_adjoint_kernel<R, CellMax<R>::T><<<v.ncell, CellMax<R>::T, smem, st>>>(v, a, 1);
    else cell_adjoint_kernel<R, 256><<<v.ncell * slices, 256, smem, st>>>(v, a, slices);
}

template <typename R>
cudaError_t set_cell_adjoint_smem_limit(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(cell_adjoint_kernel<R, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && CellMax<R>::T != 256)
        e = cudaFuncSetAttribute(cell_adjoint_kernel<R, CellMax<R>::T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

cudaError_t set_cell_adjoint_gather_smem_limit(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(cell_adjoint_gather_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cell_adjoint_gather_kernel<CellMax<float>::T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

template <typename R>
void launch_deformation_loss(const View<R> &v, const double *c0, double *cell_loss, R *dLdX, cudaStream_t st) {
    if (v.ncell == 0) return;
    deformation_loss_kernel<R><<<v.ncell, 256, 0, st>>>(v, c0, cell_loss, dLdX);
}

template void launch_cell_adjoint<double>(const View<double> &, const AdjView<double> &, cudaStream_t);
template void launch_cell_adjoint<float>(const View<float> &, const AdjView<float> &, cudaStream_t);
template cudaError_t set_cell_adjoint_smem_limit<double>(size_t);
template cudaError_t set_cell_adjoint_smem_limit<float>(size_t);
template void launch_deformation_loss<double>(const View<double> &, const double *, double *, double *, cudaStream_t);
template void launch_deformation_loss<float>(const View<float> &, const double *, double *, float *, cudaStream_t);
template void launch_cell_forces<double>(const View<double> &, int, double *, cudaStream_t);
template void launch_cell_forces<float>(const View<float> &, int, double *, cudaStream_t);
template cudaError_t set_cell_smem_limit<double>(size_t);
template cudaError_t set_cell_smem_limit<float>(size_t);

}  // namespace hemo
