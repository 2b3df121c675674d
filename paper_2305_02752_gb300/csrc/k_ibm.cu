// Immersed-boundary coupling (Sec. 2.3): vertex binning by lattice block,
// spreading of vertex forces onto the lattice and interpolation of the
// lattice velocity to the vertices with Peskin's 4-point kernel, and the
// Euler move of the vertices (Sec. 2.6).
//
// Binning: each vertex gets its stencil anchor (floor(X) per axis, wrapped on
// periodic axes, and the fraction X - floor(X)) and the key of the 8^3 block
// that holds floor(X).  Counting sort: per-block counts (warp-aggregated
// atomics), exclusive scan, scatter with per-block cursors, then each block's
// segment is ordered by vertex id, which makes the permutation the stable
// sort by (key, id) (for read-out; the step itself does not depend on the
// order of the vertices within a bin and skips that sort).
//
// Spreading in two phases without global atomics: each non-empty bin adds
// its vertices' 4x4x4 stencils into an 11^3 tile in shared memory and writes
// the tile out; then each 8^3 block (owner computes) sums the tile positions
// of its neighbouring bins that map onto its nodes and writes F = g + sum for
// every node once (no separate clearing pass).  Interpolation: one CTA per
// non-empty bin stages the velocity of its 11^3 neighbourhood in shared
// memory (FP32: one 4-D tensor copy where the neighbourhood does not wrap)
// and evaluates the 64-node stencils of its own vertices from there (FP32:
// one thread per vertex over 16-byte node records; FP64: half-warps per
// vertex, partial sums reduced with warp shuffles, several CTAs per bin).
// With the Lees-Edwards boundary the vertices whose stencil reaches across
// the plane are kept in one extra bin, handled in k_lees.cu.
#include <cstring>
#include <type_traits>

#include <cuda.h>

#include "hemo_internal.cuh"

namespace hemo {

namespace {

inline int nblocks(long long n, int b) { return (int)((n + b - 1) / b); }

__device__ __forceinline__ float sqrt_r(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqrt_r(double a) { return sqrt(a); }

constexpr int TILE = BLK + 3;           // stencil reach: one node below, two above
constexpr int TILE3 = TILE * TILE * TILE;
// Padded shared-memory strides of an 11^3 tile: the 16 lanes (b, c) of a
// half-warp address rows TS_Y*b + TS_Z*c, which fall in 16 distinct banks
// (TS_Y = 12, TS_Z = 161 = 1 mod 32).
constexpr int TS_Y = 12, TS_Z = 161;
constexpr int TILE_SMEM = TS_Z * TILE;

// A thread's walk over the positions q = l0 + TILE (l1 + TILE l2) of an
// 11^3 tile with a stride of blockDim.x: the coordinates advance by the
// stride's digits with carries, without integer division per position.
struct TileWalk {
    int l0, l1, l2, s0, s1, s2;
    __device__ __forceinline__ TileWalk(int q, int stride)
        : l0(q % TILE), l1((q / TILE) % TILE), l2(q / (TILE * TILE)), s0(stride % TILE), s1((stride / TILE) % TILE),
          s2(stride / (TILE * TILE)) {}
    __device__ __forceinline__ void next() {
        l0 += s0;
        if (l0 >= TILE) {
            l0 -= TILE;
            ++l1;
        }
        l1 += s1;
        if (l1 >= TILE) {
            l1 -= TILE;
            ++l2;
        }
        l2 += s2;
    }
};

// origin of bin k
template <typename R>
__device__ __forceinline__ void bin_origin(const View<R> &v, int k, int org[3]) {
    org[0] = (k % v.nb[0]) * BLK;
    org[1] = ((k / v.nb[0]) % v.nb[1]) * BLK;
    org[2] = (k / (v.nb[0] * v.nb[1])) * BLK;
}

template <typename R>
__global__ void anchor_count_kernel(View<R> v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.nv) return;
    const int c = v.vcell[i];
    if (!index_ok(c >= 0 && c < v.ncell, v.status)) return;
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
    // neighbouring vertex ids mostly share a block: one atomic per group
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, key);
    if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(v.counts + key, __popc(grp));
}

// exclusive scan of the block counts by one CTA of 1024 threads, over tiles
// of 4096 consecutive counts, four per thread (16-byte loads and stores
// where the arrays are 16-byte aligned; a thread's own sums, warp shuffles
// over the thread totals, the 32 warp totals by warp 0, a running carry
// between tiles; the next tile's counts are loaded before the current one
// is scanned); the counts are reset to zero for the next binning
__device__ __forceinline__ int4 load_quad(const int *p, int k, int n, bool vec) {
    if (vec && k + 3 < n) return *reinterpret_cast<const int4 *>(p + k);
    return make_int4(k < n ? p[k] : 0, k + 1 < n ? p[k + 1] : 0, k + 2 < n ? p[k + 2] : 0, k + 3 < n ? p[k + 3] : 0);
}
__device__ __forceinline__ void store_quad(int *p, int k, int n, bool vec, int4 q) {
    if (vec && k + 3 < n) {
        *reinterpret_cast<int4 *>(p + k) = q;
        return;
    }
    if (k < n) p[k] = q.x;
    if (k + 1 < n) p[k + 1] = q.y;
    if (k + 2 < n) p[k + 2] = q.z;
    if (k + 3 < n) p[k + 3] = q.w;
}
__global__ void __launch_bounds__(1024) scan_kernel(int *counts, int *start, int *cursor, int nbins) {
    __shared__ int wsum[32];
    __shared__ int carry_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const bool vec = (((uintptr_t)counts | (uintptr_t)start | (uintptr_t)cursor) & 15) == 0;
    int carry = 0;
    int4 next = load_quad(counts, 4 * t, nbins, vec);
    for (int base = 0; base < nbins; base += 4096) {
        const int k0 = base + 4 * t;
        const int4 c = next;
        if (base + 4096 < nbins) next = load_quad(counts, k0 + 4096, nbins, vec);
        const int own = c.x + c.y + c.z + c.w;
        int x = own;  // inclusive scan of the thread totals within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {  // the warp totals' inclusive scan
            int y = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            wsum[lane] = y;
            if (lane == 31) carry_s = y;
        }
        __syncthreads();
        const int e0 = carry + (w ? wsum[w - 1] : 0) + x - own;
        const int4 ex = make_int4(e0, e0 + c.x, e0 + c.x + c.y, e0 + c.x + c.y + c.z);
        store_quad(start, k0, nbins, vec, ex);
        store_quad(cursor, k0, nbins, vec, ex);
        store_quad(counts, k0, nbins, vec, make_int4(0, 0, 0, 0));
        carry += carry_s;
        __syncthreads();  // (wsum and carry_s are rewritten by the next tile)
    }
    if (t == 0) start[nbins] = carry;
}

// scatter with per-block cursors; lanes of a warp with the same key reserve
// their slots with one atomic
__global__ void scatter_kernel(const int *key, int *cursor, int *perm_raw, int nv, unsigned *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const int k = key[i];
    const int lane = threadIdx.x & 31;
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, k);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cursor + k, __popc(grp));
    base = __shfl_sync(act, base, leader);
    const int slot = base + __popc(grp & ((1u << lane) - 1u));
    if (index_ok(slot >= 0 && slot < nv, status)) perm_raw[slot] = i;
}

// One warp per block: each id's rank among the block's ids (ids are unique)
// is its position.  Segments of up to SORT_SMEM ids are ranked from shared
// memory, SORT_K ids per lane at a time held in registers (one pass over the
// segment per group); longer segments one id at a time from global memory.
constexpr int SORT_SMEM = 1024;
constexpr int SORT_K = 8;
__global__ void __launch_bounds__(128) sort_bins_kernel(const int *start, const int *perm_raw, int *perm, int nbins) {
    __shared__ int buf[4][SORT_SMEM];
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (w >= nbins) return;
    const int s = start[w], n = start[w + 1] - s;
    const int *seg = perm_raw + s;
    if (n <= SORT_SMEM) {
        for (int a = lane; a < n; a += 32) buf[wl][a] = seg[a];
        __syncwarp();
        const int *sh = buf[wl];
        for (int g0 = 0; g0 < n; g0 += 32 * SORT_K) {
            int va[SORT_K], r[SORT_K];
#pragma unroll
            for (int j = 0; j < SORT_K; ++j) {
                const int a = g0 + lane + 32 * j;
                va[j] = a < n ? sh[a] : 0x7fffffff;
                r[j] = 0;
            }
            for (int b = 0; b < n; ++b) {
                const int x = sh[b];
#pragma unroll
                for (int j = 0; j < SORT_K; ++j) r[j] += x < va[j];
            }
#pragma unroll
            for (int j = 0; j < SORT_K; ++j)
                if (g0 + lane + 32 * j < n) perm[s + r[j]] = va[j];
        }
        return;
    }
    for (int a = lane; a < n; a += 32) {
        const int va = seg[a];
        int r = 0;
        for (int b = 0; b < n; ++b) r += seg[b] < va;
        perm[s + r] = va;
    }
}

// 4-byte asynchronous copy global -> shared (completes at cp_async_wait_all)
__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// four consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void ld4v(const float *p, float *o) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    o[0] = q.x;
    o[1] = q.y;
    o[2] = q.z;
    o[3] = q.w;
}
__device__ __forceinline__ void ld4v(const double *p, double *o) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

// Peskin 4-point weights of nodes floor(X) - 1 .. floor(X) + 2 for the
// fraction t = X - floor(X) in [0, 1); one square root serves all four.
template <typename R>
__device__ __forceinline__ void peskin4(R t, R *w) {
    const R q = sqrt_r(R(1) + R(4) * t - R(4) * t * t);
    w[0] = (R(3) - R(2) * t - q) * R(0.125);
    w[1] = (R(3) - R(2) * t + q) * R(0.125);
    w[2] = (R(1) + R(2) * t + q) * R(0.125);
    w[3] = (R(1) + R(2) * t - q) * R(0.125);
}

// FP64 vertex kernels: CTAs per bin, each taking every FP64_BIN_PARTS-th
// chunk of the bin's vertices (FP64 arithmetic is slow per SM, and a bin
// crowded with vertices would otherwise keep one SM busy long after the
// others are done)
constexpr int FP64_BIN_PARTS = 8;

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

// Vertex records of one chunk of a bin, staged in shared memory: one thread
// per vertex reads its anchor through the permutation, computes its row in
// the bin's padded tile (-1 if the anchor is outside the bin, i.e. the
// vertex left the lattice) and its twelve Peskin weights (x0..3, y0..3,
// z0..3), and optionally its force (four entries per vertex, times fscale
// per component if given).  The per-vertex loops below then touch
// shared memory only.  Chunk size by precision keeps the FP64 kernels within
// 48 KB of static shared memory.
// (FP32: 240 keeps the spreading kernel at six CTAs per SM)
template <typename R> struct Stage { static constexpr int CAP = sizeof(R) == 8 ? 32 : 240; };
template <typename R>
__device__ __forceinline__ void stage_chunk(const View<R> &v, int p0, int n, const int org[3], int *srow, R *sw,
                                            R *sF, int *sperm, const R *fscale = nullptr) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int i = v.perm[p0 + j];
        if (!index_ok(i >= 0 && i < v.nv, v.status)) {
            srow[j] = -1;
            continue;
        }
        int row = 0;
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
            const int b = v.anc_i[3 * (size_t)i + d] - org[d];
            ok &= b >= 0 && b < BLK;
            row += b * (d == 0 ? 1 : (d == 1 ? TS_Y : TS_Z));
            peskin4(v.anc_t[3 * (size_t)i + d], sw + 12 * j + 4 * d);
            if (sF) sF[4 * j + d] = fscale ? v.Fv[3 * (size_t)i + d] * fscale[d] : v.Fv[3 * (size_t)i + d];
        }
        srow[j] = ok ? row : -1;
        if (sperm) sperm[j] = i;
    }
}

// Phase 1 of spreading: one CTA per non-empty bin; a warp takes two
// vertices, each half-warp's 16 lanes own one (y, z) row of the 4x4x4
// stencil and add four x-neighbours into the bin's 11^3 shared tile.  The
// tile is written out whole (compact [3][11^3]) for the owners to gather.
//
// The tile accumulates in fixed point with integer shared atomics (native,
// unaffected by address collisions, and exact: the sums do not depend on the
// order of the vertices, so every run gives the same bits).  FP32: 32-bit
// integers; per bin and component the scale is the power of two 2^e with
// e = 30 - ceil(log2(max|F| * n / 8)): a node's sum is at most max|F| times
// the sum of its n weights, each at most 1/8, so |sum| * 2^e <= 2^30, and
// the quantum, max|F| * n * 2^-33 per contribution, is below the FP32
// rounding of sums of that size.  FP64: 64-bit integers with 2^62 in place
// of 2^30 (quantum max|F| n 2^-65, below FP64 rounding).
template <typename R> struct TileAcc {
    using T = long long;
    static constexpr int E = 61;  // log2 of the bound minus one
};
template <> struct TileAcc<float> {
    using T = int;
    static constexpr int E = 29;
};
__device__ __forceinline__ int fixed_of(float x) { return __float2int_rn(x); }
__device__ __forceinline__ long long fixed_of(double x) { return __double2ll_rn(x); }

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 1) spread_tile_kernel(View<R> v) {
    using A = typename TileAcc<R>::T;
    constexpr int CAP = Stage<R>::CAP;
    const int k = blockIdx.x;
    const int s = v.start[k], e = v.start[k + 1];
    if (s == e) return;
    __shared__ A acc[3][TILE_SMEM];
    __shared__ int srow[CAP];
    __shared__ __align__(16) R sw[12 * CAP];
    __shared__ __align__(16) R sF[4 * CAP];
    __shared__ R smax[3][8];
    __shared__ R scale[3];
    for (int q = threadIdx.x; q < TILE_SMEM; q += blockDim.x) acc[0][q] = acc[1][q] = acc[2][q] = A(0);
    int org[3];
    bin_origin(v, k, org);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int h = lane >> 4, b = lane & 3, c = (lane >> 2) & 3;
    // A bin of at most CAP vertices is staged once, before the scale is known
    // (its forces unscaled; the scale is applied in the loop below, exactly,
    // being a power of two), which saves a pass over the forces; larger bins
    // take that pass first and are staged in chunks of equal size.
    const bool one = e - s <= CAP;
    if (one) stage_chunk(v, s, e - s, org, srow, sw, sF, (int *)nullptr);
    {  // one scale per component for the whole bin
        R m[3] = {R(0), R(0), R(0)};
        if (one) {
            for (int j = threadIdx.x; j < e - s; j += blockDim.x)  // (the forces this thread staged)
                for (int d = 0; d < 3; ++d) m[d] = fmax(m[d], fabs(sF[4 * j + d]));
        } else {
            for (int j = s + threadIdx.x; j < e; j += blockDim.x) {
                const int i = v.perm[j];
                if (!index_ok(i >= 0 && i < v.nv, v.status)) continue;
                for (int d = 0; d < 3; ++d) m[d] = fmax(m[d], fabs(v.Fv[3 * (size_t)i + d]));
            }
        }
        for (int d = 0; d < 3; ++d) {
            for (int o = 16; o > 0; o >>= 1) m[d] = fmax(m[d], __shfl_xor_sync(0xffffffffu, m[d], o));
            if (lane == 0) smax[d][warp] = m[d];
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            R mm = R(0);
            for (int w = 0; w < nw; ++w) mm = fmax(mm, smax[threadIdx.x][w]);
            const R bound = mm * R(e - s) * R(0.125);
            if (!(bound <= R(3.0e38))) {  // non-finite forces
                atomicOr(v.status, ST_NUMERIC);
                scale[threadIdx.x] = R(0);
            } else {
                scale[threadIdx.x] = bound > R(0) ? ldexp(R(1), min(TileAcc<R>::E - ilogb(bound), 120)) : R(0);
            }
        }
        __syncthreads();  // the staging below or the loop applies the scale
    }
    const R sc[3] = {one ? scale[0] : R(1), one ? scale[1] : R(1), one ? scale[2] : R(1)};
    const int nch = (e - s + CAP - 1) / CAP, csz = (e - s + nch - 1) / nch;
    for (int p0 = s; p0 < e; p0 += csz) {
        const int n = min(csz, e - p0);
        if (!one) {
            if (p0 != s) __syncthreads();
            stage_chunk(v, p0, n, org, srow, sw, sF, (int *)nullptr, scale);
            __syncthreads();
        }
        for (int q = 2 * warp + h; q < n; q += 2 * nw) {
            const int row0 = srow[q];
            if (row0 < 0) continue;  // vertex outside the lattice (domain status already raised)
            const R *w = sw + 12 * q;
            const R wyz = w[4 + b] * w[8 + c];
            R wx[4], fq[4];
            ld4v(w, wx);
            ld4v(sF + 4 * q, fq);  // (times the fixed-point scale, or scaled here)
            const R f[3] = {(fq[0] * sc[0]) * wyz, (fq[1] * sc[1]) * wyz, (fq[2] * sc[2]) * wyz};
            const int row = row0 + TS_Y * b + TS_Z * c;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const R wa = wx[a];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if constexpr (sizeof(A) == 4) atomicAdd((int *)&acc[d][row + a], fixed_of(f[d] * wa));
                    else atomicAdd((unsigned long long *)&acc[d][row + a], (unsigned long long)fixed_of(f[d] * wa));
                }
            }
        }
    }
    __syncthreads();
    R *out = v.tiles + (size_t)k * 3 * TILE3;
    R inv[3];
    for (int d = 0; d < 3; ++d) inv[d] = scale[d] > R(0) ? R(1) / scale[d] : R(0);  // (exact: powers of two)
    TileWalk tw(threadIdx.x, blockDim.x);
    for (int q = threadIdx.x; q < TILE3; q += blockDim.x, tw.next()) {
        const int sidx = tw.l0 + TS_Y * tw.l1 + TS_Z * tw.l2;
        for (int d = 0; d < 3; ++d) out[d * TILE3 + q] = (R)acc[d][sidx] * inv[d];
    }
}

// Phase 2 of spreading (owner computes): one CTA per 8^3 block sums, for
// each of its nodes, every tile position of the non-empty neighbouring bins
// that maps onto the node (several positions when a periodic axis is shorter
// than a tile), in a fixed order, and writes F = g + sum once.  Per axis a
// table built once per block lists, for each local coordinate, the pairs
// (neighbour slot, tile position) that land on it.
constexpr int GATHER_MAXE = 2 * TILE;  // entries per (axis, local coordinate)
template <typename R>
__global__ void __launch_bounds__(256) spread_gather_kernel(View<R> v) {
    __shared__ int nbin[27];  // bin of neighbour slot (sz*9 + sy*3 + sx), -1 if empty
    __shared__ int lb[3][3], nsl[3];
    __shared__ unsigned char cnt[3][BLK];
    __shared__ unsigned char ent_slot[3][BLK][GATHER_MAXE], ent_pos[3][BLK][GATHER_MAXE];
    const int k = blockIdx.x;
    const int bc[3] = {k % v.nb[0], (k / v.nb[0]) % v.nb[1], k / (v.nb[0] * v.nb[1])};
    const int dims[3] = {v.nx, v.ny, v.nz};
    const int t = threadIdx.x;
    if (t < 3) nsl[t] = neighbour_blocks(bc[t], v.nb[t], v.per[t], lb[t]);
    __syncthreads();
    if (t < 3 * BLK) {  // table of axis d, local coordinate l
        const int d = t / BLK, l = t % BLK;
        const int x = bc[d] * BLK + l;
        int n = 0;
        for (int sl = 0; sl < nsl[d]; ++sl) {
            const int o = lb[d][sl] * BLK - 1;  // tile origin along d
            if (v.per[d]) {
                for (int p = wrap(x - o, dims[d]); p < TILE && n < GATHER_MAXE; p += dims[d]) {
                    ent_slot[d][l][n] = (unsigned char)sl;
                    ent_pos[d][l][n++] = (unsigned char)p;
                }
            } else if (x - o >= 0 && x - o < TILE) {
                ent_slot[d][l][n] = (unsigned char)sl;
                ent_pos[d][l][n++] = (unsigned char)(x - o);
            }
        }
        cnt[d][l] = (unsigned char)n;
    } else if (t >= 32 && t < 32 + 27) {  // neighbour slot -> bin
        const int sl = t - 32, a = sl / 9, b = (sl / 3) % 3, c = sl % 3;
        int kk = -1;
        if (a < nsl[2] && b < nsl[1] && c < nsl[0]) {
            kk = lb[0][c] + v.nb[0] * (lb[1][b] + v.nb[1] * lb[2][a]);
            if (v.start[kk + 1] == v.start[kk]) kk = -1;
        }
        nbin[sl] = kk;
    }
    __syncthreads();
    const size_t N = (size_t)v.N;
    for (int q = t; q < BLK * BLK * BLK; q += blockDim.x) {
        const int l0 = q % BLK, l1 = (q / BLK) % BLK, l2 = q / (BLK * BLK);
        const int x = bc[0] * BLK + l0, y = bc[1] * BLK + l1, z = bc[2] * BLK + l2;
        if (x >= v.nx || y >= v.ny || z >= v.nz) continue;
        R f0 = R(0), f1 = R(0), f2 = R(0);
        for (int iz = 0; iz < cnt[2][l2]; ++iz)
            for (int iy = 0; iy < cnt[1][l1]; ++iy)
                for (int ix = 0; ix < cnt[0][l0]; ++ix) {
                    const int kk = nbin[9 * ent_slot[2][l2][iz] + 3 * ent_slot[1][l1][iy] + ent_slot[0][l0][ix]];
                    if (kk < 0) continue;
                    const R *tt = v.tiles + (size_t)kk * 3 * TILE3;
                    const int ti = ent_pos[0][l0][ix] + TILE * (ent_pos[1][l1][iy] + TILE * ent_pos[2][l2][iz]);
                    f0 += tt[ti];
                    f1 += tt[TILE3 + ti];
                    f2 += tt[2 * TILE3 + ti];
                }
        const size_t n = (size_t)x + (size_t)v.nx * ((size_t)y + (size_t)v.ny * z);
        const bool wall = !v.spread_all_nodes && (v.ntype[n] & 0x7f);
        v.F[n] = wall ? R(0) : v.g[0] + f0;
        v.F[N + n] = wall ? R(0) : v.g[1] + f1;
        v.F[2 * N + n] = wall ? R(0) : v.g[2] + f2;
    }
}

// Phase 2 with at least three blocks along every axis (neighbour blocks
// distinct): along an axis the lower neighbour's tile covers this block's
// local coordinates 0, 1 (tile positions 9, 10), the block's own tile all
// eight (positions 1..8) and the upper neighbour's coordinate 7 (position
// 0).  Each thread owns two nodes and adds, slot by slot in a fixed order,
// the tile values that land on them.
template <typename R>
__global__ void __launch_bounds__(256) spread_gather3_kernel(View<R> v) {
    __shared__ int nbin[27];  // bin of slot (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1), -1 if empty or absent
    const int k = blockIdx.x;
    const int bc[3] = {k % v.nb[0], (k / v.nb[0]) % v.nb[1], k / (v.nb[0] * v.nb[1])};
    const int t = threadIdx.x;
    if (t < 27) {
        const int sz = t / 9 - 1, sy = (t / 3) % 3 - 1, sx = t % 3 - 1;
        const int sl[3] = {sx, sy, sz};
        int c[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
            c[d] = bc[d] + sl[d];
            if (v.per[d]) c[d] = wrap(c[d], v.nb[d]);
            else ok &= c[d] >= 0 && c[d] < v.nb[d];
        }
        int kk = -1;
        if (ok) {
            kk = c[0] + v.nb[0] * (c[1] + v.nb[1] * c[2]);
            if (v.start[kk + 1] == v.start[kk]) kk = -1;
        }
        nbin[t] = kk;
    }
    __syncthreads();
    const size_t N = (size_t)v.N;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = t + 256 * h;
        const int l[3] = {q % BLK, (q / BLK) % BLK, q / (BLK * BLK)};
        const int x = bc[0] * BLK + l[0], y = bc[1] * BLK + l[1], z = bc[2] * BLK + l[2];
        if (x >= v.nx || y >= v.ny || z >= v.nz) continue;
        R f0 = R(0), f1 = R(0), f2 = R(0);
        // per axis: the slots reaching this coordinate and the tile position there
        int ns[3], sl[3][2] = {{0, 0}, {0, 0}, {0, 0}}, ps[3][2] = {{0, 0}, {0, 0}, {0, 0}};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // entry 0: lower neighbour (l < 2) or own block; entry 1: own block
            // (l < 2) or upper neighbour (l = 7)
            const bool lo = l[d] < 2, hi = l[d] == BLK - 1;
            sl[d][0] = lo ? 0 : 1;
            ps[d][0] = lo ? l[d] + 9 : l[d] + 1;
            sl[d][1] = lo ? 1 : 2;
            ps[d][1] = lo ? l[d] + 1 : 0;
            ns[d] = (lo || hi) ? 2 : 1;
        }
        // at most two slots per axis: fixed trip counts keep the tables in
        // registers; the tile addresses of all eight (slot x, y, z) choices
        // are formed first and the loads issued predicated, so that they are
        // all in flight together (summed in the same order, iz, iy, ix)
        const R *src[8];
        bool on[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int ix = m & 1, iy = (m >> 1) & 1, iz = m >> 2;
            const bool in = iz < ns[2] && iy < ns[1] && ix < ns[0];
            const int kk = in ? nbin[9 * sl[2][iz] + 3 * sl[1][iy] + sl[0][ix]] : -1;
            on[m] = kk >= 0;
            src[m] = v.tiles + (size_t)(kk < 0 ? 0 : kk) * 3 * TILE3 + (ps[0][ix] + TILE * (ps[1][iy] + TILE * ps[2][iz]));
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if (on[m]) {
                f0 += src[m][0];
                f1 += src[m][TILE3];
                f2 += src[m][2 * TILE3];
            }
        }
        const size_t n = (size_t)x + (size_t)v.nx * ((size_t)y + (size_t)v.ny * z);
        const bool wall = !v.spread_all_nodes && (v.ntype[n] & 0x7f);
        v.F[n] = wall ? R(0) : v.g[0] + f0;
        v.F[N + n] = wall ? R(0) : v.g[1] + f1;
        v.F[2 * N + n] = wall ? R(0) : v.g[2] + f2;
    }
}

// The move of vertex i by its interpolated velocity U (dt = 1), Sec. 2.6:
// INTEG 0 Euler; 1 Euler, keeping U; 2 the two-step Adams-Bashforth form
// with the kept velocity of the previous step, keeping U.  All loads are
// issued before the stores (off and Uprev are distinct buffers).
//
// With the adaptive separation on (v.off_eval set) it returns the vertex's
// displacement since the last force evaluation, |off - off_eval| of the new
// offsets (held steps do not re-base, so that is X - X_eval); else 0.
template <int INTEG, typename R>
__device__ __forceinline__ R move_vertex(const View<R> &v, int i, R U0, R U1, R U2) {
    R *o = v.off + 3 * (size_t)i;
    const R x0 = o[0], x1 = o[1], x2 = o[2];
    R n0, n1, n2;
    if constexpr (INTEG == 0) {
        n0 = x0 + U0;
        n1 = x1 + U1;
        n2 = x2 + U2;
    } else {
        R *p = v.Uprev + 3 * (size_t)i;
        if constexpr (INTEG == 2) {
            const R p0 = p[0], p1 = p[1], p2 = p[2];
            n0 = x0 + (R(1.5) * U0 - R(0.5) * p0);
            n1 = x1 + (R(1.5) * U1 - R(0.5) * p1);
            n2 = x2 + (R(1.5) * U2 - R(0.5) * p2);
        } else {
            n0 = x0 + U0;
            n1 = x1 + U1;
            n2 = x2 + U2;
        }
        p[0] = U0;
        p[1] = U1;
        p[2] = U2;
    }
    o[0] = n0;
    o[1] = n1;
    o[2] = n2;
    if (!v.off_eval) return R(0);
    const R *e = v.off_eval + 3 * (size_t)i;
    const R d0 = n0 - e[0], d1 = n1 - e[1], d2 = n2 - e[2];
    return sqrt_r(d0 * d0 + d1 * d1 + d2 * d2);
}

// the largest displacement of a warp's vertices into the adaptive word (as
// double bits: non-negative doubles order as their bit patterns); every
// lane calls it
__device__ __forceinline__ void adapt_max(unsigned long long *adapt, double d) {
    unsigned long long m = (unsigned long long)__double_as_longlong(d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, m, o);
        m = q > m ? q : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(adapt, m);
}

// Adaptive separation, once per step before the membrane kernels: evaluate
// the forces on the first step, when `every` steps have passed since the last
// evaluation, or when a vertex has moved more than tol since it; the
// displacement word is cleared for the coming step's interpolation.
__global__ void adapt_decide_kernel(unsigned long long *a, double tol, int every) {
    const bool eval = a[3] || a[1] >= (unsigned long long)every || __longlong_as_double((long long)a[0]) > tol;
    a[2] = eval ? 1ull : 0ull;
    a[4] += eval ? 1ull : 0ull;  // evaluations so far
    a[1] = eval ? 1ull : a[1] + 1ull;
    a[3] = 0ull;
    a[0] = 0ull;
}

// Anchors, keys and bin counts on a step between two membrane-force
// evaluations (Sec. 2.6), vertex-parallel: no re-base, so each vertex is at
// X = (hi + lo of the centroid of the last re-base) + offset.
template <typename R>
__global__ void __launch_bounds__(256) hold_bins_kernel(View<R> v) {
    if (v.adapt && v.adapt[2]) return;  // adaptive separation: this step evaluates the forces
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.nv) return;
    const int c = v.vcell[i];
    if (!index_ok(c >= 0 && c < v.ncell, v.status)) return;
    const R *cs = v.csp + 6 * (size_t)c;
    const R *o = v.off + 3 * (size_t)i;
    const R ch[3] = {cs[0], cs[1], cs[2]}, cl[3] = {cs[3], cs[4], cs[5]}, oi[3] = {o[0], o[1], o[2]};
    bin_vertex(v, (size_t)i, ch, cl, oi);
}

// Interpolation and vertex move: one CTA per non-empty bin stages u of the
// 11^3 neighbourhood in shared memory (padded strides; lattice coordinates
// of the tile's rows from per-axis tables built once); a warp takes two
// vertices, each half-warp's lanes own one (y, z) stencil row, and the 16
// partial sums are reduced with warp shuffles.
template <typename R, int INTEG>
__global__ void __launch_bounds__(256) interpolate_kernel(View<R> v, int parts) {
    drop_dead_lines(v);
    constexpr int CAP = Stage<R>::CAP;
    const int k = blockIdx.x / parts, part = blockIdx.x % parts;  // CTA part takes chunks part, part + parts, ...
    const int s = v.start[k], e = v.start[k + 1];
    if (s + part * CAP >= e) return;
    __shared__ R tile[3][TILE_SMEM];
    __shared__ int srow[CAP], sperm[CAP];
    __shared__ R sw[12 * CAP];
    __shared__ int jtab[3][TILE];  // wrapped lattice coordinate, -1 beyond a non-periodic edge
    int org[3];
    bin_origin(v, k, org);
    if (threadIdx.x < 3 * TILE) {
        const int d = threadIdx.x / TILE, l = threadIdx.x % TILE;
        const int dims = d == 0 ? v.nx : (d == 1 ? v.ny : v.nz);
        int j = org[d] - 1 + l;
        if (v.per[d]) j = wrap(j, dims);
        else if (j < 0 || j >= dims) j = -1;
        jtab[d][l] = j;
    }
    __syncthreads();
    const size_t N = (size_t)v.N;
    for (int q = threadIdx.x; q < TILE3; q += blockDim.x) {
        const int l0 = q % TILE, l1 = (q / TILE) % TILE, l2 = q / (TILE * TILE);
        const int jx = jtab[0][l0], jy = jtab[1][l1], jz = jtab[2][l2];
        const int sidx = l0 + TS_Y * l1 + TS_Z * l2;
        if ((jx | jy | jz) < 0) {  // beyond a non-periodic edge: resting wall
            tile[0][sidx] = tile[1][sidx] = tile[2][sidx] = R(0);
        } else {
            const size_t n = (size_t)jx + (size_t)v.nx * ((size_t)jy + (size_t)v.ny * jz);
            tile[0][sidx] = v.u[n];
            tile[1][sidx] = v.u[N + n];
            tile[2][sidx] = v.u[2 * N + n];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int h = lane >> 4, b = lane & 3, c = (lane >> 2) & 3;
    for (int c0 = s + part * CAP; c0 < e; c0 += parts * CAP) {
        const int n = min(CAP, e - c0);
        __syncthreads();  // the tile (first chunk) or the previous chunk's records
        stage_chunk(v, c0, n, org, srow, sw, (R *)nullptr, sperm);
        __syncthreads();
        for (int q0 = 2 * warp; q0 < n; q0 += 2 * nw) {  // uniform per warp: shuffles below
            const int q = q0 + h;
            R U0 = R(0), U1 = R(0), U2 = R(0);
            const int row0 = q < n ? srow[q] : -1;
            if (row0 >= 0) {
                const R *w = sw + 12 * q;
                const R wyz = w[4 + b] * w[8 + c];
                const int row = row0 + TS_Y * b + TS_Z * c;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const R wa = wyz * w[a];
                    U0 += wa * tile[0][row + a];
                    U1 += wa * tile[1][row + a];
                    U2 += wa * tile[2][row + a];
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                U0 += __shfl_xor_sync(0xffffffffu, U0, o);
                U1 += __shfl_xor_sync(0xffffffffu, U1, o);
                U2 += __shfl_xor_sync(0xffffffffu, U2, o);
            }
            double dmax = 0.0;
            if (row0 >= 0 && (lane & 15) == 0) dmax = move_vertex<INTEG>(v, sperm[q], U0, U1, U2);
            if (v.adapt) adapt_max(v.adapt, dmax);
        }
    }
}

// FP32 interpolation: one thread per vertex.  The bin's 11^3 neighbourhood
// of u is staged once as (ux, uy, uz, 0) per node, so each stencil node is
// one 16-byte shared load; the weights stay in registers and each thread
// sums its vertex's 64 terms itself (no staging of weights, no shuffles).
//
// Staging.  With a tensor map of u (4-D: x, y, z, component) one thread
// copies the box x in [ox - 4, ox + 12), y in [oy - 1, oy + 10), z in
// [oz - 1, oz + 10), all three components, into shared memory with a single
// tensor copy (x starts 16-byte aligned: ox is a multiple of 8; coordinates
// outside the lattice read as zero, the resting wall beyond a non-periodic
// edge); the threads then rearrange it into the node records, in place (each
// first reads its nodes' values into registers).  A bin whose neighbourhood
// wraps around a periodic edge, and every bin without a tensor map, is
// staged node by node with 4-byte asynchronous copies.
constexpr int IT_Y = TILE, IT_Z = TILE * TILE;  // node record strides of the interpolation tile
constexpr int UBOX_X = 16;                      // x extent of the tensor copy (nodes)
constexpr unsigned UBOX_BYTES = 3u * UBOX_X * TILE * TILE * 4u;
constexpr int INTERP_SMEM = UBOX_BYTES > 16u * TILE3 ? (int)UBOX_BYTES : 16 * TILE3;
__device__ __forceinline__ void tma_load_4d(void *dst, const void *map, int c0, int c1, int c2, int c3, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

template <int INTEG>
__global__ void __launch_bounds__(256, 6) interpolate_v4_kernel(View<float> v, const __grid_constant__ CUtensorMap umap) {
    drop_dead_lines(v);
    const int k = blockIdx.x;
    const int s = v.start[k], e = v.start[k + 1];
    if (s == e) return;
    __shared__ __align__(128) unsigned char tile_raw[INTERP_SMEM];
    __shared__ int jtab[3][TILE];  // wrapped lattice coordinate, -1 beyond a non-periodic edge
    __shared__ __align__(8) uint64_t bar;
    float4 *tile = reinterpret_cast<float4 *>(tile_raw);
    int org[3];
    bin_origin(v, k, org);
    // the tensor copy serves a neighbourhood that does not wrap
    bool boxed = v.u_tmap != nullptr;
    for (int d = 0; d < 3; ++d) {
        const int dims = d == 0 ? v.nx : (d == 1 ? v.ny : v.nz);
        if (v.per[d] && (org[d] - 1 < 0 || org[d] + BLK + 1 >= dims)) boxed = false;
    }
    if (boxed && v.stalled_wait_test) {
        // failure-path test: wait on a barrier that nothing arrives at (no
        // copy issued); the bounded wait runs out and the CTA reports it
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        const bool ok = threadIdx.x == 0 ? mbar_wait(&bar, 0u, 2000000ull) : true;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(v.status, ST_TIMEOUT);
            return;
        }
    }
    if (boxed && threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        fence_async_smem();
        mbar_expect_tx(&bar, UBOX_BYTES);
        tma_load_4d(tile_raw, &umap, org[0] - 4, org[1] - 1, org[2] - 1, 0, &bar);
    }
    // this thread's first vertex: its records are requested before the tile
    // is staged, so their latency overlaps the staging
    const int jf = s + threadIdx.x;
    int ifst = -1, aif[3] = {0, 0, 0};
    float atf[3] = {0.f, 0.f, 0.f};
    if (jf < e) {
        ifst = v.perm[jf];
        if (!index_ok(ifst >= 0 && ifst < v.nv, v.status)) ifst = -1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            aif[d] = ifst < 0 ? 0 : v.anc_i[3 * (size_t)ifst + d];
            atf[d] = ifst < 0 ? 0.f : v.anc_t[3 * (size_t)ifst + d];
        }
    }
    if (boxed) {
        __syncthreads();  // (the barrier is initialised)
        const bool ok = mbar_wait(&bar, 0);
        if (__syncthreads_or(!ok)) {  // the copy did not complete in time: report, let it land, leave
            if (threadIdx.x == 0) {
                atomicOr(v.status, ST_TIMEOUT);
                mbar_wait(&bar, 0);
            }
            __syncthreads();
            return;
        }
        // rearrange [component][z][y][x - ox + 4] into node records, in place
        constexpr int PER = (TILE3 + 255) / 256;
        const float *box = reinterpret_cast<const float *>(tile_raw);
        float4 r[PER];
        TileWalk tw(threadIdx.x, blockDim.x);
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int q = threadIdx.x + 256 * m;
            if (q < TILE3) {
                const int b0 = tw.l0 + 3 + UBOX_X * (tw.l1 + TILE * tw.l2);
                r[m] = make_float4(box[b0], box[b0 + UBOX_X * TILE * TILE], box[b0 + 2 * UBOX_X * TILE * TILE], 0.f);
            }
            tw.next();
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int q = threadIdx.x + 256 * m;
            if (q < TILE3) tile[q] = r[m];
        }
    } else {
        if (threadIdx.x < 3 * TILE) {
            const int d = threadIdx.x / TILE, l = threadIdx.x % TILE;
            const int dims = d == 0 ? v.nx : (d == 1 ? v.ny : v.nz);
            int j = org[d] - 1 + l;
            if (v.per[d]) j = wrap(j, dims);
            else if (j < 0 || j >= dims) j = -1;
            jtab[d][l] = j;
        }
        __syncthreads();
        const size_t N = (size_t)v.N;
        // asynchronous copies (no register round trip: all of a thread's loads
        // are in flight at once); nodes beyond a non-periodic edge are a
        // resting wall
        for (int q = threadIdx.x; q < TILE3; q += blockDim.x) {
            const int l0 = q % TILE, l1 = (q / TILE) % TILE, l2 = q / (TILE * TILE);
            const int jx = jtab[0][l0], jy = jtab[1][l1], jz = jtab[2][l2];
            float4 *dst = tile + q;
            if ((jx | jy | jz) >= 0) {
                const size_t n = (size_t)jx + (size_t)v.nx * ((size_t)jy + (size_t)v.ny * jz);
                cp_async4(&dst->x, v.u + n);
                cp_async4(&dst->y, v.u + N + n);
                cp_async4(&dst->z, v.u + 2 * N + n);
            } else {
                *dst = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();
    float dmax = 0.f;  // adaptive separation: this thread's largest displacement
    for (int j = jf; j < e; j += blockDim.x) {
        int i;
        int ai[3];
        float at[3];
        if (j == jf) {
            i = ifst;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                ai[d] = aif[d];
                at[d] = atf[d];
            }
        } else {
            i = v.perm[j];
            if (!index_ok(i >= 0 && i < v.nv, v.status)) continue;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                ai[d] = v.anc_i[3 * (size_t)i + d];
                at[d] = v.anc_t[3 * (size_t)i + d];
            }
        }
#if HEMO_BOUNDS_CHECK
        if (i < 0) continue;  // (a vertex id that failed its check)
#endif
        // the move's loads (offsets; the previous velocity for Adams-Bashforth;
        // the offsets of the last force evaluation for the adaptive
        // separation) are requested into L1 before the stencil sums, whose
        // shared loads would otherwise hide nothing of their latency
        prefetch_l1(v.off + 3 * (size_t)i);
        if (INTEG == 2) prefetch_l1(v.Uprev + 3 * (size_t)i);
        if (v.off_eval) prefetch_l1(v.off_eval + 3 * (size_t)i);
        float w[3][4];
        int r0 = 0;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int b = ai[d] - org[d];
            ok &= b >= 0 && b < BLK;
            r0 += b * (d == 0 ? 1 : (d == 1 ? IT_Y : IT_Z));
            peskin4(at[d], w[d]);
        }
        if (!ok) continue;
        float U0 = 0.f, U1 = 0.f, U2 = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float wyz = w[1][b] * w[2][c];
                const float4 *row = tile + r0 + IT_Y * b + IT_Z * c;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float wa = wyz * w[0][a];
                    const float4 t = row[a];
                    U0 += wa * t.x;
                    U1 += wa * t.y;
                    U2 += wa * t.z;
                }
            }
        dmax = fmaxf(dmax, move_vertex<INTEG>(v, i, U0, U1, U2));
    }
    if (v.adapt) adapt_max(v.adapt, (double)dmax);  // (FP64 once per thread, adaptive runs only)
}

// Peskin weights and their derivatives d/dt for the fraction t
template <typename R>
__device__ __forceinline__ void peskin4_d(R t, R *w, R *dw) {
    const R q = sqrt_r(R(1) + R(4) * t - R(4) * t * t);
    const R qp = (R(2) - R(4) * t) / q;
    w[0] = (R(3) - R(2) * t - q) * R(0.125);
    w[1] = (R(3) - R(2) * t + q) * R(0.125);
    w[2] = (R(1) + R(2) * t + q) * R(0.125);
    w[3] = (R(1) + R(2) * t - q) * R(0.125);
    dw[0] = (R(-2) - qp) * R(0.125);
    dw[1] = (R(-2) + qp) * R(0.125);
    dw[2] = (R(2) + qp) * R(0.125);
    dw[3] = (R(2) - qp) * R(0.125);
}

// Adjoint of the coupling operators at the vertices (differentiation form):
// for each vertex v of a bin, with the lattice field A staged like the
// velocity in interpolate_kernel,
//   out_interp[v]  = sum_x w(X_v, x) A(x)                  (interpolation)
//   out_grad[v]   += sum_x (A(x) . B[v]) grad_X w(X_v, x)  (position derivative)
// grad_X w = (w'_x w_y w_z, w_x w'_y w_z, w_x w_y w'_z).  Either output may
// be null (B is then unused).  out_grad may alias B: a vertex reads B[v]
// before its own write.
template <typename R> struct VfStage { static constexpr int CAP = sizeof(R) == 8 ? 16 : 128; };
template <typename R>
__global__ void __launch_bounds__(256) vertex_field_kernel(View<R> v, const R *A, const R *B, R *out_grad,
                                                           R *out_interp, int parts) {
    constexpr int CAP = VfStage<R>::CAP;
    const int k = blockIdx.x / parts, part = blockIdx.x % parts;  // CTA part takes chunks part, part + parts, ...
    const int s = v.start[k], e = v.start[k + 1];
    if (s + part * CAP >= e) return;
    __shared__ R tile[3][TILE_SMEM];
    __shared__ int srow[CAP], sperm[CAP];
    __shared__ R sw[24 * CAP], sB[3 * CAP];
    __shared__ int jtab[3][TILE];
    int org[3];
    bin_origin(v, k, org);
    if (threadIdx.x < 3 * TILE) {
        const int d = threadIdx.x / TILE, l = threadIdx.x % TILE;
        const int dims = d == 0 ? v.nx : (d == 1 ? v.ny : v.nz);
        int j = org[d] - 1 + l;
        if (v.per[d]) j = wrap(j, dims);
        else if (j < 0 || j >= dims) j = -1;
        jtab[d][l] = j;
    }
    __syncthreads();
    const size_t N = (size_t)v.N;
    for (int q = threadIdx.x; q < TILE3; q += blockDim.x) {
        const int l0 = q % TILE, l1 = (q / TILE) % TILE, l2 = q / (TILE * TILE);
        const int jx = jtab[0][l0], jy = jtab[1][l1], jz = jtab[2][l2];
        const int sidx = l0 + TS_Y * l1 + TS_Z * l2;
        if ((jx | jy | jz) < 0) {
            tile[0][sidx] = tile[1][sidx] = tile[2][sidx] = R(0);
        } else {
            const size_t n = (size_t)jx + (size_t)v.nx * ((size_t)jy + (size_t)v.ny * jz);
            tile[0][sidx] = A[n];
            tile[1][sidx] = A[N + n];
            tile[2][sidx] = A[2 * N + n];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int h = lane >> 4, b = lane & 3, c = (lane >> 2) & 3;
    for (int c0 = s + part * CAP; c0 < e; c0 += parts * CAP) {
        const int n = min(CAP, e - c0);
        __syncthreads();  // the tile (first chunk) or the previous chunk's records
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const int i = v.perm[c0 + j];
            int row = 0;
            bool ok = true;
            for (int d = 0; d < 3; ++d) {
                const int bb = v.anc_i[3 * (size_t)i + d] - org[d];
                ok &= bb >= 0 && bb < BLK;
                row += bb * (d == 0 ? 1 : (d == 1 ? TS_Y : TS_Z));
                peskin4_d(v.anc_t[3 * (size_t)i + d], sw + 24 * j + 4 * d, sw + 24 * j + 12 + 4 * d);
                sB[3 * j + d] = B ? B[3 * (size_t)i + d] : R(0);
            }
            srow[j] = ok ? row : -1;
            sperm[j] = i;
        }
        __syncthreads();
        for (int q0 = 2 * warp; q0 < n; q0 += 2 * nw) {  // uniform per warp: shuffles below
            const int q = q0 + h;
            R U[3] = {R(0), R(0), R(0)}, G[3] = {R(0), R(0), R(0)};
            const int row0 = q < n ? srow[q] : -1;
            if (row0 >= 0) {
                const R *w = sw + 24 * q, *dw = w + 12;
                const R Bv[3] = {sB[3 * q], sB[3 * q + 1], sB[3 * q + 2]};
                const R wy = w[4 + b], wz = w[8 + c], dwy = dw[4 + b], dwz = dw[8 + c];
                const int row = row0 + TS_Y * b + TS_Z * c;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const R A0 = tile[0][row + a], A1 = tile[1][row + a], A2 = tile[2][row + a];
                    const R wxyz = w[a] * wy * wz;
                    U[0] += wxyz * A0;
                    U[1] += wxyz * A1;
                    U[2] += wxyz * A2;
                    const R sAB = A0 * Bv[0] + A1 * Bv[1] + A2 * Bv[2];
                    G[0] += sAB * dw[a] * wy * wz;
                    G[1] += sAB * w[a] * dwy * wz;
                    G[2] += sAB * w[a] * wy * dwz;
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1)
                for (int d = 0; d < 3; ++d) {
                    U[d] += __shfl_xor_sync(0xffffffffu, U[d], o);
                    G[d] += __shfl_xor_sync(0xffffffffu, G[d], o);
                }
            if (row0 >= 0 && (lane & 15) == 0) {
                const size_t vid = (size_t)sperm[q];
                for (int d = 0; d < 3; ++d) {
                    if (out_interp) out_interp[3 * vid + d] = U[d];
                    if (out_grad) out_grad[3 * vid + d] += G[d];
                }
            }
        }
    }
}

// FP32 form of vertex_field_kernel: one thread per vertex over a float4
// tile, as in interpolate_v4_kernel
__global__ void __launch_bounds__(256) vertex_field_v4_kernel(View<float> v, const float *A, const float *B,
                                                              float *out_grad, float *out_interp) {
    const int k = blockIdx.x;
    const int s = v.start[k], e = v.start[k + 1];
    if (s == e) return;
    __shared__ float4 tile[TILE_SMEM];
    __shared__ int jtab[3][TILE];
    int org[3];
    bin_origin(v, k, org);
    if (threadIdx.x < 3 * TILE) {
        const int d = threadIdx.x / TILE, l = threadIdx.x % TILE;
        const int dims = d == 0 ? v.nx : (d == 1 ? v.ny : v.nz);
        int j = org[d] - 1 + l;
        if (v.per[d]) j = wrap(j, dims);
        else if (j < 0 || j >= dims) j = -1;
        jtab[d][l] = j;
    }
    __syncthreads();
    const size_t N = (size_t)v.N;
    for (int q = threadIdx.x; q < TILE3; q += blockDim.x) {
        const int l0 = q % TILE, l1 = (q / TILE) % TILE, l2 = q / (TILE * TILE);
        const int jx = jtab[0][l0], jy = jtab[1][l1], jz = jtab[2][l2];
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((jx | jy | jz) >= 0) {
            const size_t n = (size_t)jx + (size_t)v.nx * ((size_t)jy + (size_t)v.ny * jz);
            t.x = A[n];
            t.y = A[N + n];
            t.z = A[2 * N + n];
        }
        tile[l0 + TS_Y * l1 + TS_Z * l2] = t;
    }
    __syncthreads();
    for (int j = s + threadIdx.x; j < e; j += blockDim.x) {
        const int i = v.perm[j];
        float w[3][4], dw[3][4];
        int r0 = 0;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int b = v.anc_i[3 * (size_t)i + d] - org[d];
            ok &= b >= 0 && b < BLK;
            r0 += b * (d == 0 ? 1 : (d == 1 ? TS_Y : TS_Z));
            peskin4_d(v.anc_t[3 * (size_t)i + d], w[d], dw[d]);
        }
        if (!ok) continue;
        const float B0 = B ? B[3 * (size_t)i] : 0.f, B1 = B ? B[3 * (size_t)i + 1] : 0.f, B2 = B ? B[3 * (size_t)i + 2] : 0.f;
        float U0 = 0.f, U1 = 0.f, U2 = 0.f, G0 = 0.f, G1 = 0.f, G2 = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float wyz = w[1][b] * w[2][c], dyz = dw[1][b] * w[2][c], ydz = w[1][b] * dw[2][c];
                const float4 *row = tile + r0 + TS_Y * b + TS_Z * c;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float4 t = row[a];
                    const float wa = w[0][a] * wyz;
                    U0 += wa * t.x;
                    U1 += wa * t.y;
                    U2 += wa * t.z;
                    const float sAB = t.x * B0 + t.y * B1 + t.z * B2;
                    G0 += sAB * dw[0][a] * wyz;
                    G1 += sAB * w[0][a] * dyz;
                    G2 += sAB * w[0][a] * ydz;
                }
            }
        if (out_interp) {
            out_interp[3 * (size_t)i] = U0;
            out_interp[3 * (size_t)i + 1] = U1;
            out_interp[3 * (size_t)i + 2] = U2;
        }
        if (out_grad) {
            out_grad[3 * (size_t)i] += G0;
            out_grad[3 * (size_t)i + 1] += G1;
            out_grad[3 * (size_t)i + 2] += G2;
        }
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
void launch_bins(const View<R> &v, cudaStream_t st, bool stable) {
    cudaMemsetAsync(v.counts, 0, sizeof(int) * v.nbins, st);
    anchor_count_kernel<R><<<nblocks(v.nv, 256), 256, 0, st>>>(v);
    scan_kernel<<<1, 1024, 0, st>>>(v.counts, v.start, v.cursor, v.nbins);
    if (stable) {
        scatter_kernel<<<nblocks(v.nv, 256), 256, 0, st>>>(v.key, v.cursor, v.perm_raw, v.nv, v.status);
        sort_bins_kernel<<<nblocks((long long)v.nbins * 32, 128), 128, 0, st>>>(v.start, v.perm_raw, v.perm, v.nbins);
    } else {
        scatter_kernel<<<nblocks(v.nv, 256), 256, 0, st>>>(v.key, v.cursor, v.perm, v.nv, v.status);
    }
}

template <typename R>
void launch_bin_ranges(const View<R> &v, cudaStream_t st) {
    scan_kernel<<<1, 1024, 0, st>>>(v.counts, v.start, v.cursor, v.nbins + (v.le ? 1 : 0));  // (+ the Lees-Edwards bin)
    scatter_kernel<<<nblocks(v.nv, 256), 256, 0, st>>>(v.key, v.cursor, v.perm, v.nv, v.status);
}

template <typename R>
void launch_spread(const View<R> &v, cudaStream_t st) {
    spread_tile_kernel<R><<<v.nbins, 256, 0, st>>>(v);
    if (v.nb[0] >= 3 && v.nb[1] >= 3 && v.nb[2] >= 3) spread_gather3_kernel<R><<<v.nbins, 256, 0, st>>>(v);
    else spread_gather_kernel<R><<<v.nbins, 256, 0, st>>>(v);
}

template <typename R, int INTEG>
void launch_interpolate_as(const View<R> &v, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value) {
        // the tensor map describes the step's u array only (the adjoint's
        // recomputation keeps u per step elsewhere)
        View<float> w = v;
        CUtensorMap map;
        if (v.u_tmap && v.u_tmap_base == (const void *)v.u) {
            std::memcpy(&map, v.u_tmap, sizeof(map));
        } else {
            std::memset(&map, 0, sizeof(map));
            w.u_tmap = nullptr;
        }
        interpolate_v4_kernel<INTEG><<<v.nbins, 256, 0, st>>>(w, map);
    }
    else interpolate_kernel<R, INTEG><<<v.nbins * FP64_BIN_PARTS, 256, 0, st>>>(v, FP64_BIN_PARTS);
}

template <typename R>
void launch_interpolate(const View<R> &v, cudaStream_t st) {
    if (v.integ == 2) launch_interpolate_as<R, 2>(v, st);
    else if (v.integ == 1) launch_interpolate_as<R, 1>(v, st);
    else launch_interpolate_as<R, 0>(v, st);
}

template <typename R>
void launch_hold_bins(const View<R> &v, cudaStream_t st) {
    if (v.nv) hold_bins_kernel<R><<<nblocks(v.nv, 256), 256, 0, st>>>(v);
}

void launch_adapt_decide(unsigned long long *adapt, double tol, int every, cudaStream_t st) {
    adapt_decide_kernel<<<1, 1, 0, st>>>(adapt, tol, every);
}

template <typename R>
void launch_vertex_field(const View<R> &v, const R *field, const R *vec, R *out_grad, R *out_interp, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value)
        vertex_field_v4_kernel<<<v.nbins, 256, 0, st>>>(v, field, vec, out_grad, out_interp);
    else
        vertex_field_kernel<R><<<v.nbins * FP64_BIN_PARTS, 256, 0, st>>>(v, field, vec, out_grad, out_interp, FP64_BIN_PARTS);
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
    template void launch_bins<R>(const View<R> &, cudaStream_t, bool);                    \
    template void launch_bin_ranges<R>(const View<R> &, cudaStream_t);                     \
    template void launch_spread<R>(const View<R> &, cudaStream_t);                        \
    template void launch_interpolate<R>(const View<R> &, cudaStream_t);                   \
    template void launch_hold_bins<R>(const View<R> &, cudaStream_t);                     \
    template void launch_verts_out<R>(const View<R> &, double *, double *, cudaStream_t); \
    template void launch_vertex_field<R>(const View<R> &, const R *, const R *, R *, R *, cudaStream_t); \
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
    // block counts in 64 bits; each factor is checked before the product so
    // that no intermediate can overflow
    const long long nb0 = (long long)nx / BLK + (nx % BLK != 0), nb1 = (long long)ny / BLK + (ny % BLK != 0),
                    nb2 = (long long)nz / BLK + (nz % BLK != 0);
    if (nb0 > NOALLOC_MAX_BINS || nb1 > NOALLOC_MAX_BINS || nb2 > NOALLOC_MAX_BINS || nb0 * nb1 > NOALLOC_MAX_BINS ||
        nb0 * nb1 * nb2 > NOALLOC_MAX_BINS)
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
        scatter_kernel<<<(nv + 255) / 256, 256, 0, st>>>(key, cursor, perm_raw, nv, nullptr);
        sort_bins_kernel<<<(int)(((long long)nbins * 32 + 127) / 128), 128, 0, st>>>(start, perm_raw, perm, nbins);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(HEMO_ERR_CUDA, cudaGetErrorString(e));
    return HEMO_OK;
}
