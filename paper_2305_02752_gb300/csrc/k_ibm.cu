// Immersed-boundary coupling (Sec. 2.3): vertex binning by lattice block,
// spreading of vertex forces onto the lattice and interpolation of the
// lattice velocity to the vertices with Peskin's 4-point kernel, and the
// Euler move of the vertices (Sec. 2.6).
//
// Binning: each vertex gets its stencil anchor (floor(X) per axis, wrapped on
// periodic axes, and the fraction X - floor(X)) and the key of the 8^3 block
// that holds floor(X).  Counting sort: per-block counts, exclusive scan,
// scatter with per-block cursors, then each block's segment is ordered by
// vertex id, which makes the permutation the stable sort by (key, id).
//
// Spreading is owner-computes: one CTA per lattice block gathers the
// vertices of the (up to 27) neighbouring blocks, adds the parts of their
// 4x4x4 stencils that fall inside its own 8^3 nodes into shared memory, and
// writes F = g + sum for every node of the block once (no global atomics, no
// separate clearing pass).  Interpolation: one CTA per non-empty block stages
// the velocity of its 11^3 neighbourhood in shared memory and evaluates the
// 64-node stencils of its own vertices from there.
#include "hemo_internal.cuh"

namespace hemo {

namespace {

inline int nblocks(long long n, int b) { return (int)((n + b - 1) / b); }

__device__ __forceinline__ float sqrt_r(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqrt_r(double a) { return sqrt(a); }

// Peskin 4-point weights of nodes floor(X) - 1 .. floor(X) + 2 for the
// fraction t = X - floor(X) in [0, 1); one square root serves all four.
template <typename R>
__device__ __forceinline__ void peskin4(R t, R w[4]) {
    const R q = sqrt_r(R(1) + R(4) * t - R(4) * t * t);
    w[0] = (R(3) - R(2) * t - q) * R(0.125);
    w[1] = (R(3) - R(2) * t + q) * R(0.125);
    w[2] = (R(1) + R(2) * t + q) * R(0.125);
    w[3] = (R(1) + R(2) * t - q) * R(0.125);
}

template <typename R>
__global__ void anchor_count_kernel(View<R> v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.nv) return;
    const int c = v.vcell[i];
    const int dims[3] = {v.nx, v.ny, v.nz};
    int b[3];
    for (int d = 0; d < 3; ++d) {
        const double X = v.ctr[3 * c + d] + (double)v.off[3 * (size_t)i + d];
        const double fl = floor(X);
        int j = (int)fl;
        const R t = R(X - fl);
        if (v.per[d]) {
            j = wrap(j, dims[d]);
        } else if (!(X >= 0.0 && X < (double)dims[d])) {
            atomicOr(v.status, ST_DOMAIN);
        }
        v.anc_i[3 * (size_t)i + d] = j;
        v.anc_t[3 * (size_t)i + d] = t;
        const int jc = j < 0 ? 0 : (j >= dims[d] ? dims[d] - 1 : j);
        b[d] = jc / BLK;
    }
    const int key = b[0] + v.nb[0] * (b[1] + v.nb[1] * b[2]);
    v.key[i] = key;
    atomicAdd(v.counts + key, 1);
}

// exclusive scan of the block counts by one CTA of 1024 threads
__global__ void __launch_bounds__(1024) scan_kernel(const int *counts, int *start, int *cursor, int nbins) {
    __shared__ int part[1024];
    const int per = (nbins + 1023) / 1024;
    const int lo = threadIdx.x * per;
    const int hi = min(lo + per, nbins);
    int s = 0;
    for (int k = lo; k < hi; ++k) s += counts[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
        const int add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int k = lo; k < hi; ++k) {
        start[k] = run;
        cursor[k] = run;
        run += counts[k];
    }
    if (threadIdx.x == 1023) start[nbins] = part[1023];
}

__global__ void scatter_kernel(const int *key, int *cursor, int *perm_raw, int nv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    perm_raw[atomicAdd(cursor + key[i], 1)] = i;
}

// one warp per block: rank each id among the block's ids (ids are unique)
__global__ void sort_bins_kernel(const int *start, const int *perm_raw, int *perm, int nbins) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nbins) return;
    const int s = start[w], n = start[w + 1] - s;
    const int *seg = perm_raw + s;
    for (int a = lane; a < n; a += 32) {
        const int va = seg[a];
        int r = 0;
        for (int b = 0; b < n; ++b) r += seg[b] < va;
        perm[s + r] = va;
    }
}

template <typename R>
__global__ void gather_kernel(View<R> v) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.nv) return;
    const int i = v.perm[p];
    for (int d = 0; d < 3; ++d) {
        v.s_i[3 * (size_t)p + d] = v.anc_i[3 * (size_t)i + d];
        v.s_t[3 * (size_t)p + d] = v.anc_t[3 * (size_t)i + d];
        v.s_F[3 * (size_t)p + d] = v.Fv[3 * (size_t)i + d];
    }
}

// distinct neighbour block coordinates along one axis
__device__ __forceinline__ int neighbour_blocks(int b, int nb, int periodic, int out[3]) {
    int cnt = 0;
    for (int d = -1; d <= 1; ++d) {
        int q = b + d;
        if (periodic) q = wrap(q, nb);
        else if (q < 0 || q >= nb) continue;
        bool dup = false;
        for (int k = 0; k < cnt; ++k) dup |= out[k] == q;
        if (!dup) out[cnt++] = q;
    }
    return cnt;
}

template <typename R>
__global__ void __launch_bounds__(256) spread_kernel(View<R> v) {
    __shared__ R acc[3][BLK * BLK * BLK];
    __shared__ int seg_s[27], seg_pre[28];
    __shared__ int nseg;
    const int k = blockIdx.x;
    const int bx = k % v.nb[0], by = (k / v.nb[0]) % v.nb[1], bz = k / (v.nb[0] * v.nb[1]);
    const int org[3] = {bx * BLK, by * BLK, bz * BLK};
    const int dims[3] = {v.nx, v.ny, v.nz};
    for (int q = threadIdx.x; q < BLK * BLK * BLK; q += blockDim.x) acc[0][q] = acc[1][q] = acc[2][q] = R(0);
    if (threadIdx.x == 0) {
        int lx[3], ly[3], lz[3];
        const int ncx = neighbour_blocks(bx, v.nb[0], v.per[0], lx);
        const int ncy = neighbour_blocks(by, v.nb[1], v.per[1], ly);
        const int ncz = neighbour_blocks(bz, v.nb[2], v.per[2], lz);
        int ns = 0, run = 0;
        for (int a = 0; a < ncz; ++a)
            for (int b = 0; b < ncy; ++b)
                for (int c = 0; c < ncx; ++c) {
                    const int kk = lx[c] + v.nb[0] * (ly[b] + v.nb[1] * lz[a]);
                    const int s0 = v.start[kk], s1 = v.start[kk + 1];
                    if (s1 == s0) continue;
                    seg_s[ns] = s0;
                    seg_pre[ns] = run;
                    run += s1 - s0;
                    ++ns;
                }
        seg_pre[ns] = run;
        nseg = ns;
    }
    __syncthreads();
    const int total = seg_pre[nseg];
    int seg = 0;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        while (q >= seg_pre[seg + 1]) ++seg;
        const size_t p = (size_t)seg_s[seg] + (q - seg_pre[seg]);
        R w[3][4];
        int l[3][4];
        bool any = true;
        for (int d = 0; d < 3 && any; ++d) {
            const int i0 = v.s_i[3 * p + d];
            peskin4(v.s_t[3 * p + d], w[d]);
            bool hit = false;
            for (int a = 0; a < 4; ++a) {
                int j = i0 + a - 1;
                if (v.per[d]) j = wrap(j, dims[d]);
                const int lj = j - org[d];
                const bool in = lj >= 0 && lj < BLK && j < dims[d] && j >= 0;
                l[d][a] = in ? lj : -1;
                hit |= in;
            }
            any = hit;
        }
        if (!any) continue;
        const R Fx = v.s_F[3 * p], Fy = v.s_F[3 * p + 1], Fz = v.s_F[3 * p + 2];
        for (int c = 0; c < 4; ++c) {
            if (l[2][c] < 0) continue;
            for (int b = 0; b < 4; ++b) {
                if (l[1][b] < 0) continue;
                const R wzy = w[2][c] * w[1][b];
                for (int a = 0; a < 4; ++a) {
                    if (l[0][a] < 0) continue;
                    const R ww = wzy * w[0][a];
                    const int idx = l[0][a] + BLK * (l[1][b] + BLK * l[2][c]);
                    atomicAdd(&acc[0][idx], Fx * ww);
                    atomicAdd(&acc[1][idx], Fy * ww);
                    atomicAdd(&acc[2][idx], Fz * ww);
                }
            }
        }
    }
    __syncthreads();
    const size_t N = (size_t)v.N;
    for (int q = threadIdx.x; q < BLK * BLK * BLK; q += blockDim.x) {
        const int x = org[0] + (q % BLK), y = org[1] + (q / BLK) % BLK, z = org[2] + q / (BLK * BLK);
        if (x >= v.nx || y >= v.ny || z >= v.nz) continue;
        const size_t n = (size_t)x + (size_t)v.nx * ((size_t)y + (size_t)v.ny * z);
        const bool wall = v.ntype[n] & 0x7f;
        v.F[n] = wall ? R(0) : v.g[0] + acc[0][q];
        v.F[N + n] = wall ? R(0) : v.g[1] + acc[1][q];
        v.F[2 * N + n] = wall ? R(0) : v.g[2] + acc[2][q];
    }
}

constexpr int TILE = BLK + 3;  // stencil reach: one node below, two above

template <typename R>
__global__ void __launch_bounds__(256) interpolate_kernel(View<R> v) {
    const int k = blockIdx.x;
    const int s = v.start[k], e = v.start[k + 1];
    if (s == e) return;
    __shared__ R tile[3][TILE * TILE * TILE];
    const int bx = k % v.nb[0], by = (k / v.nb[0]) % v.nb[1], bz = k / (v.nb[0] * v.nb[1]);
    const int org[3] = {bx * BLK, by * BLK, bz * BLK};
    const int dims[3] = {v.nx, v.ny, v.nz};
    const size_t N = (size_t)v.N;
    for (int q = threadIdx.x; q < TILE * TILE * TILE; q += blockDim.x) {
        int j[3] = {org[0] - 1 + q % TILE, org[1] - 1 + (q / TILE) % TILE, org[2] - 1 + q / (TILE * TILE)};
        bool out = false;
        for (int d = 0; d < 3; ++d) {
            if (v.per[d]) j[d] = wrap(j[d], dims[d]);
            else out |= j[d] < 0 || j[d] >= dims[d];
        }
        if (out) {  // beyond a non-periodic edge: resting wall
            tile[0][q] = tile[1][q] = tile[2][q] = R(0);
        } else {
            const size_t n = (size_t)j[0] + (size_t)v.nx * ((size_t)j[1] + (size_t)v.ny * j[2]);
            tile[0][q] = v.u[n];
            tile[1][q] = v.u[N + n];
            tile[2][q] = v.u[2 * N + n];
        }
    }
    __syncthreads();
    for (int p = s + threadIdx.x; p < e; p += blockDim.x) {
        R w[3][4];
        int base[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
            base[d] = v.s_i[3 * (size_t)p + d] - org[d];  // stencil starts at tile index base
            ok &= base[d] >= 0 && base[d] < BLK;
            peskin4(v.s_t[3 * (size_t)p + d], w[d]);
        }
        if (!ok) continue;  // vertex outside the lattice (domain status already raised)
        R U[3] = {R(0), R(0), R(0)};
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b) {
                const R wzy = w[2][c] * w[1][b];
                const int row = (base[0]) + TILE * ((base[1] + b) + TILE * (base[2] + c));
                for (int a = 0; a < 4; ++a) {
                    const R ww = wzy * w[0][a];
                    U[0] += ww * tile[0][row + a];
                    U[1] += ww * tile[1][row + a];
                    U[2] += ww * tile[2][row + a];
                }
            }
        const int vid = v.perm[p];
        R *o = v.off + 3 * (size_t)vid;
        o[0] += U[0];
        o[1] += U[1];
        o[2] += U[2];
    }
}

template <typename R>
__global__ void verts_out_kernel(View<R> v, double *X, double *F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.nv) return;
    const int c = v.vcell[i];
    for (int d = 0; d < 3; ++d) {
        if (X) X[3 * (size_t)i + d] = v.ctr[3 * c + d] + (double)v.off[3 * (size_t)i + d];
        if (F) F[3 * (size_t)i + d] = (double)v.Fv[3 * (size_t)i + d];
    }
}

template <typename R>
__global__ void set_vertices_kernel(View<R> v, const double *X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.nv) return;
    const int c = v.vcell[i];
    for (int d = 0; d < 3; ++d) v.off[3 * (size_t)i + d] = R(X[3 * (size_t)i + d] - v.ctr[3 * c + d]);
}

}  // namespace

template <typename R>
void launch_bins(const View<R> &v, cudaStream_t st) {
    cudaMemsetAsync(v.counts, 0, sizeof(int) * v.nbins, st);
    anchor_count_kernel<R><<<nblocks(v.nv, 256), 256, 0, st>>>(v);
    scan_kernel<<<1, 1024, 0, st>>>(v.counts, v.start, v.cursor, v.nbins);
    scatter_kernel<<<nblocks(v.nv, 256), 256, 0, st>>>(v.key, v.cursor, v.perm_raw, v.nv);
    sort_bins_kernel<<<nblocks((long long)v.nbins * 32, 128), 128, 0, st>>>(v.start, v.perm_raw, v.perm, v.nbins);
}

template <typename R>
void launch_gather(const View<R> &v, cudaStream_t st) {
    gather_kernel<R><<<nblocks(v.nv, 256), 256, 0, st>>>(v);
}

template <typename R>
void launch_spread(const View<R> &v, cudaStream_t st) {
    spread_kernel<R><<<v.nbins, 256, 0, st>>>(v);
}

template <typename R>
void launch_interpolate(const View<R> &v, cudaStream_t st) {
    interpolate_kernel<R><<<v.nbins, 256, 0, st>>>(v);
}

template <typename R>
void launch_verts_out(const View<R> &v, double *X, double *F, cudaStream_t st) {
    if (v.nv) verts_out_kernel<R><<<nblocks(v.nv, 256), 256, 0, st>>>(v, X, F);
}

template <typename R>
void launch_set_vertices(const View<R> &v, const double *X, cudaStream_t st) {
    if (v.nv) set_vertices_kernel<R><<<nblocks(v.nv, 256), 256, 0, st>>>(v, X);
}

#define HEMO_INST(R)                                                                      \
    template void launch_bins<R>(const View<R> &, cudaStream_t);                          \
    template void launch_gather<R>(const View<R> &, cudaStream_t);                        \
    template void launch_spread<R>(const View<R> &, cudaStream_t);                        \
    template void launch_interpolate<R>(const View<R> &, cudaStream_t);                   \
    template void launch_verts_out<R>(const View<R> &, double *, double *, cudaStream_t); \
    template void launch_set_vertices<R>(const View<R> &, const double *, cudaStream_t);
HEMO_INST(double)
HEMO_INST(float)

}  // namespace hemo

// ===========================================================================
// Vertex binning without any device allocation.
//
// Some callers cannot let a library allocate device memory: code that runs
// inside another framework's memory budget (a caching allocator that owns
// all of the GPU's memory), latency-critical loops in which cudaMalloc's
// implicit device synchronisation is not acceptable, or tools that hold
// vertex positions in their own buffers and no simulation handle.  For them
// hemo_bin_vertices_noalloc runs the same binning kernels as the step on
// caller-owned inputs and outputs, with its scratch (block counts, block
// cursors, unsorted permutation) in the file-scope array below.  The array
// is part of the loaded module: every GPU that loads the library holds its
// 5 MiB until the process exits.
// ===========================================================================
#include <mutex>

namespace hemo {

namespace {

constexpr int NOALLOC_MAX_VERTICES = 1 << 20;  // 1,048,576 vertices
constexpr int NOALLOC_MAX_BINS = 1 << 17;      // 131,072 blocks of 8^3 nodes

// [0, MAX_BINS): counts; [MAX_BINS, 2 MAX_BINS): cursors; then the unsorted
// permutation (MAX_VERTICES entries)
static __device__ __align__(256) int g_bin_scratch[2 * NOALLOC_MAX_BINS + NOALLOC_MAX_VERTICES];

// Device address of g_bin_scratch per device; in host code the symbol is
// only a host-side stand-in, so its address is taken once per device with
// cudaGetSymbolAddress while that device is current.
constexpr int NOALLOC_MAX_DEVICES = 64;
int *g_bin_scratch_dev[NOALLOC_MAX_DEVICES] = {};
std::mutex g_bin_scratch_mutex;

// key and count of each vertex from absolute FP64 positions (same floor,
// wrap and clamp rule as the step's anchor kernel)
__global__ void abs_key_count_kernel(const double *X, int nv, int nx, int ny, int nz, int px, int py, int pz,
                                     int nb0, int nb1, int *key, int *counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const int dims[3] = {nx, ny, nz};
    const int per[3] = {px, py, pz};
    int b[3];
    for (int d = 0; d < 3; ++d) {
        int j = (int)floor(X[3 * (size_t)i + d]);
        if (per[d]) j = wrap(j, dims[d]);
        const int jc = j < 0 ? 0 : (j >= dims[d] ? dims[d] - 1 : j);
        b[d] = jc / BLK;
    }
    const int k = b[0] + nb0 * (b[1] + nb1 * b[2]);
    key[i] = k;
    atomicAdd(counts + k, 1);
}

int noalloc_fail(int code, const char *msg) {
    set_last_error(msg);  // reported by hemo_last_error()
    return code;
}

}  // namespace

}  // namespace hemo

extern "C" int hemo_bin_vertices_noalloc(const double *verts, int nv, int nx, int ny, int nz, const int32_t *periodic,
                                         int32_t *key, int32_t *perm, int32_t *start, void *cuda_stream) {
    using namespace hemo;
    if (nx < 1 || ny < 1 || nz < 1 || nv < 0 || !periodic || !start || (nv > 0 && (!verts || !key || !perm)))
        return noalloc_fail(HEMO_ERR_ARG, "hemo_bin_vertices_noalloc: bad sizes or null pointer");
    if (nv > NOALLOC_MAX_VERTICES)
        return noalloc_fail(HEMO_ERR_ARG, "hemo_bin_vertices_noalloc: more than 1,048,576 vertices");
    const long long nb0 = (nx + BLK - 1) / BLK, nb1 = (ny + BLK - 1) / BLK, nb2 = (nz + BLK - 1) / BLK;
    if (nb0 * nb1 * nb2 > NOALLOC_MAX_BINS)
        return noalloc_fail(HEMO_ERR_ARG, "hemo_bin_vertices_noalloc: more than 131,072 lattice blocks of 8^3 nodes");
    const int nbins = (int)(nb0 * nb1 * nb2);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return noalloc_fail(HEMO_ERR_CUDA, "hemo_bin_vertices_noalloc: no usable current device");
    int *scratch;
    {
        std::lock_guard<std::mutex> lock(g_bin_scratch_mutex);
        if (!g_bin_scratch_dev[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
            if (e != cudaSuccess || !p) return noalloc_fail(HEMO_ERR_CUDA, "hemo_bin_vertices_noalloc: cudaGetSymbolAddress failed");
            g_bin_scratch_dev[dev] = (int *)p;
        }
        scratch = g_bin_scratch_dev[dev];
    }
    int *counts = scratch, *cursor = scratch + NOALLOC_MAX_BINS, *perm_raw = scratch + 2 * NOALLOC_MAX_BINS;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: the counts must start at zero
    if (cudaMemsetAsync(counts, 0, sizeof(int) * nbins, st) != cudaSuccess)
        return noalloc_fail(HEMO_ERR_CUDA, "hemo_bin_vertices_noalloc: clearing the counts failed");
    if (nv > 0)
        abs_key_count_kernel<<<(nv + 255) / 256, 256, 0, st>>>(verts, nv, nx, ny, nz, periodic[0] != 0, periodic[1] != 0,
                                                               periodic[2] != 0, (int)nb0, (int)nb1, key, counts);
    scan_kernel<<<1, 1024, 0, st>>>(counts, start, cursor, nbins);
    if (nv > 0) {
        scatter_kernel<<<(nv + 255) / 256, 256, 0, st>>>(key, cursor, perm_raw, nv);
        sort_bins_kernel<<<(int)(((long long)nbins * 32 + 127) / 128), 128, 0, st>>>(start, perm_raw, perm, nbins);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(HEMO_ERR_CUDA, cudaGetErrorString(e));
    return HEMO_OK;
}
