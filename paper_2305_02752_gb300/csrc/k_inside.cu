// Inside/outside indicator of the cell membranes for the internal viscosity
// (Sec. 1: the cytosol is five times as viscous as the plasma; Sec. 3: the
// red-cell model carries an internal viscosity ratio).
//
// A node is inside when the upward ray from it crosses the membrane with a
// net signed count of one (sign of the outward normal's z component).
// Equivalently, scanning a lattice column (x, y) upwards, the count of the
// cells a node is in changes by -sign at every crossing at or below it.  So:
//   1. one CTA per cell: each triangle finds the lattice columns inside its
//      xy-projection (an edge shared by two triangles is evaluated in one
//      canonical vertex order so both agree on the columns it passes
//      through; a column exactly on an edge belongs to the triangle for which
//      the edge, counter-clockwise seen from +z, points in -y, or in +x when
//      horizontal) and adds -sign at the first node at or above the crossing
//      height, atomically, into a per-node toggle count;
//   2. the toggles of each column are summed upwards (segments of the column
//      in parallel); on a periodic z axis a cell may wrap around, and the
//      column's count is the running sum minus its minimum (a column always
//      passes outside every cell somewhere).  The indicator is count > 0; the
//      toggles are reset for the next step.
#include "hemo_internal.cuh"

namespace hemo {

namespace {

// twice the signed area of the xy-projection of edge u -> v against the point
// (px, py), computed from the lower-numbered vertex
template <typename R>
__device__ __forceinline__ R edge_fn(const R (*P)[3], const int *id, int u, int w, R px, R py) {
    if (id[u] < id[w]) return (P[w][0] - P[u][0]) * (py - P[u][1]) - (P[w][1] - P[u][1]) * (px - P[u][0]);
    return -((P[u][0] - P[w][0]) * (py - P[w][1]) - (P[u][1] - P[w][1]) * (px - P[w][0]));
}

// one thread per triangle: grid (cells, triangle blocks of 256)
template <typename R>
__global__ void __launch_bounds__(256) inside_toggle_kernel(View<R> v) {
    const int c = blockIdx.x;
    const MeshDev<R> m = v.meshes[v.cell_type[c]];
    const int first = v.cell_first[c];
    const int dims[3] = {v.nx, v.ny, v.nz};
    const double C[3] = {v.ctr[3 * c], v.ctr[3 * c + 1], v.ctr[3 * c + 2]};
    {
        const int t = blockIdx.y * blockDim.x + threadIdx.x;
        if (t >= m.nt) return;
        int id[3];
        R P[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            id[k] = m.tri[3 * t + k];
            const R *o = v.off + 3 * (size_t)(first + id[k]);
#pragma unroll
            for (int d = 0; d < 3; ++d) P[k][d] = R(C[d]) + o[d];  // absolute position
        }
        // outward normal n = (P1 - P0) x (P2 - P0)
        const R e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
        const R e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
        const R nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2], nz = e1[0] * e2[1] - e1[1] * e2[0];
        if (nz == R(0)) return;
        const int sgn = nz > R(0) ? 1 : -1;
        // corners counter-clockwise seen from +z
        const int o0 = 0, o1 = sgn > 0 ? 1 : 2, o2 = sgn > 0 ? 2 : 1;
        const int ord[3] = {o0, o1, o2};
        R lo[2], hi[2];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            lo[d] = fmin(P[0][d], fmin(P[1][d], P[2][d]));
            hi[d] = fmax(P[0][d], fmax(P[1][d], P[2][d]));
        }
        const int jx0 = (int)ceil(lo[0]), jx1 = (int)floor(hi[0]);
        const int jy0 = (int)ceil(lo[1]), jy1 = (int)floor(hi[1]);
        for (int jy = jy0; jy <= jy1; ++jy)
            for (int jx = jx0; jx <= jx1; ++jx) {
                const R px = R(jx), py = R(jy);
                bool in = true;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int u = ord[k], w = ord[(k + 1) % 3];
                    const R e = edge_fn(P, id, u, w, px, py);
                    if (e < R(0)) in = false;
                    else if (e == R(0)) {
                        const R dx = P[w][0] - P[u][0], dy = P[w][1] - P[u][1];
                        if (!(dy < R(0) || (dy == R(0) && dx > R(0)))) in = false;
                    }
                }
                if (!in) continue;
                const R zc = P[0][2] - (nx * (px - P[0][0]) + ny * (py - P[0][1])) / nz;
                int kz = (int)ceil(zc);
                int qx = jx, qy = jy;
                if (v.per[0]) qx = wrap(qx, dims[0]);
                else if (qx < 0 || qx >= dims[0]) continue;
                if (v.per[1]) qy = wrap(qy, dims[1]);
                else if (qy < 0 || qy >= dims[1]) continue;
                if (v.per[2]) {
                    kz = wrap(kz, dims[2]);
                } else {
                    if (kz >= dims[2]) continue;  // above every node of the column
                    if (kz < 0) kz = 0;
                }
                atomicAdd(v.tog + (size_t)qx + (size_t)v.nx * ((size_t)qy + (size_t)v.ny * kz), -sgn);
            }
    }
}

// 32 consecutive columns (x) per CTA, their z range split into SCAN_G
// segments: each thread sums its segment (loads coalesced across the x
// lanes), the segment offsets and the column minimum come from shared
// memory, then each thread writes its segment's indicator.
constexpr int SCAN_G = 8;
template <typename R>
__global__ void __launch_bounds__(32 * SCAN_G) inside_scan_kernel(View<R> v) {
    __shared__ int ssum[SCAN_G][32], smin[SCAN_G][32];
    const int lx = threadIdx.x, g = threadIdx.y;
    const int x = blockIdx.x * 32 + lx, y = blockIdx.y;
    const bool col_ok = x < v.nx;
    const size_t stride = (size_t)v.nx * v.ny;
    const size_t base = (size_t)x + (size_t)v.nx * y;
    const int seg = (v.nz + SCAN_G - 1) / SCAN_G, z0 = g * seg, z1 = min(v.nz, z0 + seg);
    int p = 0, mn = 0;
    if (col_ok)
        for (int z = z0; z < z1; ++z) {
            p += v.tog[base + stride * z];
            mn = min(mn, p);
        }
    ssum[g][lx] = p;
    smin[g][lx] = mn;
    __syncthreads();
    // running sum before this segment, and the column minimum (at least 0:
    // the count before z = 0 is the starting point)
    int off = 0, cmin = 0, run = 0;
    for (int k = 0; k < SCAN_G; ++k) {
        if (k == g) off = run;
        cmin = min(cmin, run + smin[k][lx]);
        run += ssum[k][lx];
    }
    if (!col_ok) return;
    p = off - cmin;  // the count just below z0
    for (int z = z0; z < z1; ++z) {
        const size_t n = base + stride * z;
        p += v.tog[n];
        v.tog[n] = 0;
        v.ind[n] = p > 0 ? 1 : 0;
    }
}

}  // namespace

template <typename R>
void launch_inside(const View<R> &v, cudaStream_t st) {
    if (v.ncell) inside_toggle_kernel<R><<<dim3(v.ncell, (v.max_nt + 255) / 256), 256, 0, st>>>(v);
    inside_scan_kernel<R><<<dim3((v.nx + 31) / 32, v.ny), dim3(32, SCAN_G), 0, st>>>(v);
}

template void launch_inside<double>(const View<double> &, cudaStream_t);
template void launch_inside<float>(const View<float> &, cudaStream_t);

}  // namespace hemo
