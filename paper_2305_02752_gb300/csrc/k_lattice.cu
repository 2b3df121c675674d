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
//
// 16-bit storage subtracts a per-row reference equilibrium from what it
// stores (see row_refs below) and collides two nodes per thread
// (collide_pair_kernel).
#include <type_traits>

#include "lattice_core.cuh"

namespace hemo {

namespace {

// ---------------------------------------------------------------------------
// Reference equilibrium of 16-bit storage.
//
// A 2-byte population keeps 8 (BF16) or 11 (FP16) significant bits of what
// is stored, so what is stored should be small.  Each row (x-line, index
// r = y + ny z) has a reference x-velocity U_r, and a population of
// direction i with cx_i != 0 held in a slot of row r is stored as
//   f_i - w_i - K_i(r),   K_i(r) = w_i (3 cx_i U_r + 3 U_r^2),
// which is f_i^eq(1, (U_r, 0, 0)) - w_i for those directions; for cx_i = 0
// that equilibrium deviation is -1.5 w_i U_r^2, small, and nothing is
// subtracted.  In a flow near the rows' reference profile what is stored
// is the non-equilibrium part and the departure from the profile.  Per row
// the table holds P = (3 U + 3 U^2) / 18 and M = (-3 U + 3 U^2) / 18 (the
// axis weight; diagonals take half).  The reference belongs to the slot
// that holds the value: the kernel that writes a slot and the one that
// reads it use the same row's reference, so decoding is exact but for the
// FP32 rounding of one addition.  In natural order slot i of node n holds
// direction i arriving at n (row of n); after an even step slot opp(i) of n
// holds direction i leaving n (row of n).  With a zero table (no reference)
// the stored values are the plain deviations f_i - w_i.
// ---------------------------------------------------------------------------
template <typename T> struct HasRef { static constexpr bool value = sizeof(T) == 2; };

// K_i of a row from its (P, M)
__device__ __forceinline__ float ref_dir(int i, float2 pm) {
    if (cx(i) == 0) return 0.f;
    const float k = cx(i) > 0 ? pm.x : pm.y;
    return (cy(i) != 0 || cz(i) != 0) ? 0.5f * k : k;
}

// (P, M) of a node's row and of the rows y -/+ 1 and z -/+ 1 (wrapped: a
// wrapped row is used only across a periodic edge, a non-periodic edge
// being a wall link)
struct RowRefs {
    float2 own, ym, yp, zm, zp;
    // the row displaced by (dy, dz), at most one of them nonzero
    __device__ __forceinline__ float2 at(int dy, int dz) const {
        return dy > 0 ? yp : (dy < 0 ? ym : (dz > 0 ? zp : (dz < 0 ? zm : own)));
    }
};

template <typename T, typename R>
__device__ __forceinline__ RowRefs row_refs(const View<R> &v, int y, int z, bool neighbours) {
    RowRefs r;
    if constexpr (HasRef<T>::value) {
        const float2 *t = v.rref;
        const int ny = v.ny, row = y + ny * z;
        r.own = t[row];
        if (neighbours) {
            r.ym = t[row + (y == 0 ? ny - 1 : -1)];
            r.yp = t[row + (y == ny - 1 ? 1 - ny : 1)];
            r.zm = t[z == 0 ? row + ny * (v.nz - 1) : row - ny];
            r.zp = t[z == v.nz - 1 ? y : row + ny];
        } else {
            r.ym = r.yp = r.zm = r.zp = r.own;
        }
    } else {
        r.own = r.ym = r.yp = r.zm = r.zp = make_float2(0.f, 0.f);
    }
    return r;
}

template <typename T, typename R>
__device__ __forceinline__ RowRefs row_refs_of(const View<R> &v, int n, bool neighbours) {
    const int r = n / v.nx;
    return row_refs<T>(v, r % v.ny, r / v.ny, neighbours);
}

// decode / encode one stored value with the reference `ref` of its slot;
// has_ref false (directions with cx_i = 0, whose reference is zero): the
// value as stored, without adding the zero
template <typename T, typename R>
__device__ __forceinline__ R dec(T s, float ref, bool has_ref) {
    if constexpr (HasRef<T>::value) return has_ref ? Store<T>::ld(s) + ref : Store<T>::ld(s);
    else return Store<T>::ld(s);
}
template <typename T, typename R>
__device__ __forceinline__ T enc(R q, float ref) {
    if constexpr (HasRef<T>::value) return Store<T>::st(q - ref);
    else return Store<T>::st(q);
}

// Read the 19 populations arriving at node n.  LAYOUT 0: natural order (slot
// i of n).  LAYOUT 1: after an even step (slot opp(i) of n - c_i, or slot i
// of n when n - c_i is a wall).  LINKS false: no wall among the neighbours
// (lk is not read).  I: the index type of the population array, 32-bit
// unsigned when 19 N < 2^32 (fewer registers and address instructions).
template <typename T, typename R, int LAYOUT, bool LINKS, typename I = size_t>
__device__ __forceinline__ void load_pops(const View<R> &v, int n, uint64_t lk, const Nbr &o, const RowRefs &rr,
                                          R d[Q]) {
    const T *f = (const T *)v.f;
    const I N = (I)v.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (LAYOUT == 0) {
            d[i] = dec<T, R>(f[(I)i * N + (I)n], ref_dir(i, rr.own), cx(i) != 0);
        } else {
            if (i == 0) {
                d[i] = dec<T, R>(f[n], 0.f, false);
            } else if (LINKS && link_code(lk, opp(i))) {  // slot i holds direction opp(i) leaving n
                d[i] = dec<T, R>(f[(I)i * N + (I)n], ref_dir(opp(i), rr.own), cx(i) != 0);
            } else {  // direction i leaving n - c_i
                d[i] = dec<T, R>(f[(I)opp(i) * N + (I)(n + o.of(-cx(i), -cy(i), -cz(i)))],
                                 ref_dir(i, rr.at(-cy(i), -cz(i))), cx(i) != 0);
            }
        }
    }
}

// collision and streaming of fluid node n with neighbour offsets o,
// reading and writing the global array directly; LINKS false for a node
// without wall neighbours (most of them: that path carries no wall terms)
template <typename T, typename R, int PARITY, bool LINKS, typename I, bool VISC = true>
__device__ __forceinline__ void collide_core(const View<R> &v, int n, const Nbr &o, uint64_t lk, const RowRefs &rr) {
    R d[Q], p[Q];
    load_pops<T, R, PARITY, LINKS, I>(v, n, lk, o, rr, d);
    const size_t N = (size_t)v.N;
    R rho, ux, uy, uz;
    const R om = (VISC && v.ind && v.ind[n]) ? v.omega_in : v.omega;  // inside a cell: internal viscosity
    bgk_guo<R>(d, v.F[n], v.F[N + n], v.F[2 * N + n], om, p, rho, ux, uy, uz);
    if (v.rec) {
        v.rec[n] = rho;
        v.rec[N + n] = ux;
        v.rec[2 * N + n] = uy;
        v.rec[3 * N + n] = uz;
    }
    T *f = (T *)v.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int code = LINKS ? link_code(lk, i) : 0;
        R q = p[i];
        if (code) {
            const R cw = R(cx(i)) * v.uw[code][0] + R(cy(i)) * v.uw[code][1] + R(cz(i)) * v.uw[code][2];
            q -= R(6) * R(wgt(i)) * rho * cw;
        }
        const I NI = (I)N;
        if (PARITY == 0) {  // slot opp(i) of n: direction i leaving n
            f[(I)opp(i) * NI + (I)n] = enc<T, R>(q, ref_dir(i, rr.own));
        } else {
            if (code)  // bounced back: direction opp(i) arriving at n
                f[(I)opp(i) * NI + (I)n] = enc<T, R>(q, ref_dir(opp(i), rr.own));
            else  // direction i arriving at n + c_i
                f[(I)i * NI + (I)(n + o.of(cx(i), cy(i), cz(i)))] = enc<T, R>(q, ref_dir(i, rr.at(cy(i), cz(i))));
        }
    }
}

// node (x, y, z) = index n; VISC: the internal viscosity may be on
template <typename T, typename R, int PARITY, typename I, bool VISC>
__device__ __forceinline__ void collide_at(const View<R> &v, int n, int x, int y, int z) {
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) return;  // wall node
    const RowRefs rr = row_refs<T>(v, y, z, PARITY == 1);
    if (nt & 0x80) collide_core<T, R, PARITY, true, I, VISC>(v, n, nbr_at(v, x, y, z), v.links[n], rr);
    else collide_core<T, R, PARITY, false, I, VISC>(v, n, nbr_at(v, x, y, z), 0ull, rr);
}

// any node given by its index (walls included), one code path for nodes
// with and without wall links (the rows next to walls)
template <typename T, typename R, int PARITY, typename I>
__device__ __forceinline__ void collide_node(const View<R> &v, int n) {
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) return;  // wall node
    const int r = n / v.nx, y = r % v.ny, z = r / v.ny;
    collide_core<T, R, PARITY, true, I>(v, n, nbr_at(v, n % v.nx, y, z), (nt & 0x80) ? v.links[n] : 0ull,
                                        row_refs<T>(v, y, z, PARITY == 1));
}

// all nodes, grid of NODE_BX x NODE_BY blocks over (x, y, z)
template <typename T, typename R, int PARITY, typename I, bool VISC>
__global__ void __launch_bounds__(NODE_BX * NODE_BY, sizeof(R) == 4 ? 4 : 1) collide_stream_kernel(View<R> v) {
    drop_dead_lines(v);
    const int x = blockIdx.x * NODE_BX + threadIdx.x, y = blockIdx.y * NODE_BY + threadIdx.y, z = blockIdx.z;
    if (x >= v.nx || y >= v.ny) return;
    collide_at<T, R, PARITY, I, VISC>(v, x + v.nx * (y + v.ny * z), x, y, z);
}

// ---------------------------------------------------------------------------
// Staged collision for tiles of interior rows.
//
// An interior row is an x-line whose nodes, and the nodes of the eight rows
// around it, are all fluid (x periodic): no population of its nodes meets a
// wall.  For such a tile of consecutive rows, the 19 slot ranges that its
// nodes read in one step are whole rows, and every element of those ranges is
// read and written by exactly one node of the tile (even step: slot i of the
// tile's own rows; odd step: slot opp(i) of the rows shifted by -c_i, the
// x-shift applied in shared memory with the periodic wrap).  One persistent
// CTA per SM runs a ring of up to four shared-memory stages of 1024 nodes:
// a producer warp copies a tile's 19 ranges and its force rows into a stage
// by bulk copies (cp.async.bulk, completion on the stage's "full" mbarrier),
// the consumer warps collide in place (each node writes its outgoing value
// where the opposite incoming value was) and arrive on the stage's "empty"
// mbarrier, and the producer writes the same ranges back by bulk stores and
// refills the stage.  The consumers never wait on the producer's issue of
// copies, only on data, and up to three stages of loads are in flight while
// they compute the fourth, without holding them in registers (what 2-byte
// populations need to reach the HBM bandwidth).  A second kernel
// (collide_erows_kernel) collides the rows next to walls node by node.
constexpr int TILE_NODES = 1024;           // stride of a direction's range in a stage (nodes)
constexpr int TILE_CONSUMER_WARPS = 18;
constexpr int TILE_THREADS = 32 * (1 + TILE_CONSUMER_WARPS);  // warp 0: the producer
constexpr int TILE_MAX_STAGES = 4;

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int K>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(K) : "memory");
}

// The rows of a tile (k rows from row (y0, z) of the lattice) shifted by
// (dy, dz), as at most two contiguous pieces (a periodic wrap in y splits
// them): fn(first element of the piece in the lattice, first element in the
// tile buffer, element count).
template <typename R, typename Fn>
__device__ __forceinline__ void tile_pieces(const View<R> &v, int y0, int z, int k, int dy, int dz, Fn fn) {
    const long long plane = (long long)v.ny * wrap(z + dz, v.nz);
    const int ya = wrap(y0 + dy, v.ny);
    const int c1 = min(k, v.ny - ya);
    fn((plane + ya) * v.nx, 0, c1 * v.nx);
    if (c1 < k) fn(plane * v.nx, c1 * v.nx, (k - c1) * v.nx);
}

// y and z components of the velocities packed two bits each (c + 1), so
// that lanes holding different directions look them up without a table
__host__ __device__ constexpr unsigned long long pack_c(int axis) {
    unsigned long long b = 0;
    for (int i = 0; i < Q; ++i) b |= (unsigned long long)((axis == 1 ? cy(i) : cz(i)) + 1) << (2 * i);
    return b;
}
constexpr unsigned long long CY_PACK = pack_c(1), CZ_PACK = pack_c(2);
__device__ __forceinline__ int cy_of(int i) { return (int)((CY_PACK >> (2 * i)) & 3ull) - 1; }
__device__ __forceinline__ int cz_of(int i) { return (int)((CZ_PACK >> (2 * i)) & 3ull) - 1; }
static_assert(((CY_PACK >> 6) & 3) == 2 && ((CZ_PACK >> 10) & 3) == 2, "packed velocity components");

constexpr int TILE_COPIES = Q + 3;  // lanes of the producer warp that issue the copies of a stage

template <typename T, typename R, int PARITY, typename I>
__global__ void __launch_bounds__(TILE_THREADS, 1) collide_tiles_kernel(View<R> v) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);  // [stage]: the stage's copies have landed
    uint64_t *empty = full + TILE_MAX_STAGES;             // [stage]: the consumers are done with it
    uint64_t *test_bar = empty + TILE_MAX_STAGES;
    unsigned char *ring = smem + 128;
    constexpr int TNM = TILE_NODES;
    constexpr size_t pop_bytes = (size_t)TNM * sizeof(T), stage_bytes = Q * pop_bytes + 3 * (size_t)TNM * sizeof(R);
    const int nx = v.nx, S = v.tile_stages;
    const size_t N = (size_t)v.N;
    const int ntiles = v.ntiles;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    auto tile_of = [&](int it) { return (int)blockIdx.x + it * (int)gridDim.x; };
    T *f = (T *)v.f;

    drop_dead_lines(v);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full + s, TILE_COPIES);
            mbar_init(empty + s, TILE_CONSUMER_WARPS);
        }
        mbar_init(test_bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (v.stalled_wait_test) {
        // failure-path test: wait on a barrier that nothing arrives at; the
        // bounded wait runs out and the kernel reports it without touching
        // the populations (no copy has been issued)
        const bool ok = threadIdx.x == 0 ? mbar_wait(test_bar, 0u, 2000000ull) : true;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(v.status, ST_TIMEOUT);
            return;
        }
    }

    if (warp == 0) {
        // Producer.  Lane i < 19 copies direction i's range (slot i of the
        // tile's rows on even steps, slot opp(i) of the rows shifted by -c_i
        // on odd steps) and writes it back; lanes 19..21 copy the three force
        // components.  Each lane announces its own bytes on the stage's full
        // barrier (22 arrivals).
        const bool issuer = lane < TILE_COPIES, storer = lane < Q;
        auto issue_load = [&](int it) {
            const int4 tl = v.rtiles[tile_of(it)];
            const int s = it % S;
            unsigned char *st = ring + s * stage_bytes;
            const unsigned tn = (unsigned)(tl.y * nx);
            if (lane < Q) {
                T *buf = (T *)(st + lane * pop_bytes);
                const T *src = f + (size_t)(PARITY ? opp(lane) : lane) * N;
                mbar_expect_tx(full + s, tn * (unsigned)sizeof(T));
                tile_pieces(v, tl.z, tl.w, tl.y, PARITY ? -cy_of(lane) : 0, PARITY ? -cz_of(lane) : 0,
                            [&](long long g, int b, int cnt) {
                                bulk_load(buf + b, src + g, (unsigned)(cnt * sizeof(T)), full + s);
                            });
            } else {
                const int c = lane - Q;
                R *fs = (R *)(st + Q * pop_bytes) + c * TNM;
                mbar_expect_tx(full + s, tn * (unsigned)sizeof(R));
                bulk_load(fs, v.F + c * N + (size_t)tl.x * nx, tn * (unsigned)sizeof(R), full + s);
            }
        };
        auto issue_store = [&](int it) {  // lane < 19: the range it loaded
            const int4 tl = v.rtiles[tile_of(it)];
            unsigned char *st = ring + (it % S) * stage_bytes;
            T *buf = (T *)(st + lane * pop_bytes);
            T *dst = f + (size_t)(PARITY ? opp(lane) : lane) * N;
            tile_pieces(v, tl.z, tl.w, tl.y, PARITY ? -cy_of(lane) : 0, PARITY ? -cz_of(lane) : 0,
                        [&](long long g, int b, int cnt) { bulk_store(dst + g, buf + b, (unsigned)(cnt * sizeof(T))); });
            bulk_commit();
        };
        // wait until the consumers are done with tile j, then write it back
        // (every lane waits, so that the whole warp agrees on the outcome)
        auto retire = [&](int j) {
            const bool ok = mbar_wait(empty + j % S, (unsigned)((j / S) & 1));
            if (!__all_sync(0xffffffffu, ok)) return false;
            if (storer) issue_store(j);
            return true;
        };
        bool ok = true;
        int it = 0;
        for (; tile_of(it) < ntiles; ++it) {
            if (it >= S) {  // the stage of tile it held tile it - S
                if (!(ok = retire(it - S))) break;
                if (storer) bulk_wait_read<0>();  // its stores have read the stage
                __syncwarp();
            }
            if (issuer) issue_load(it);
        }
        for (int j = it - S < 0 ? 0 : it - S; ok && j < it; ++j) ok = retire(j);
        if (!ok) {
            // a wait ran out (a consumer gave up): report, and let every load
            // issued into a stage land before the CTA ends
            if (lane == 0) {
                atomicOr(v.status, ST_TIMEOUT);
                for (int j = it - S < 0 ? 0 : it - S; j < it; ++j) mbar_wait(full + j % S, (unsigned)((j / S) & 1));
            }
            __syncwarp();
        }
        if (storer) bulk_wait_read<0>();
        return;
    }

    // Consumers: the nodes of a tile (row j, column x) spread over all
    // consumer threads; this thread's first node (j0, x0) and the step to
    // its next one (dj, dx), taken once
    constexpr int CT = 32 * TILE_CONSUMER_WARPS;
    const int ct = threadIdx.x - 32;
    const int x0 = ct % nx, j0 = ct / nx, dx = CT % nx, dj = CT / nx;
    // the tile table entry is read one tile ahead, and the references of
    // the thread's first row before the wait for the stage's data, so that
    // their latency overlaps the wait
    int4 tl = tile_of(0) < ntiles ? v.rtiles[tile_of(0)] : make_int4(0, 0, 0, 0);
    for (int it = 0; tile_of(it) < ntiles; ++it) {
        const int s = it % S;
        const int4 tl_next = tile_of(it + 1) < ntiles ? v.rtiles[tile_of(it + 1)] : tl;
        const int y0 = tl.z, z0 = tl.w;  // a tile's rows lie in one z-plane
        // the node's row and its neighbours' references (direction i arrives
        // from the row shifted by -c_i and leaves to the row shifted by
        // +c_i), reloaded when the row changes
        int rj = j0 < tl.y ? j0 : tl.y - 1;
        RowRefs rr = row_refs<T>(v, y0 + rj, z0, PARITY == 1);
        const bool ok = mbar_wait(full + s, (unsigned)((it / S) & 1));
        if (!__all_sync(0xffffffffu, ok)) {  // the producer's copies did not land in time
            if (lane == 0) atomicOr(v.status, ST_TIMEOUT);
            return;
        }
        T *P = (T *)(ring + s * stage_bytes);
        const R *Fs = (const R *)(ring + s * stage_bytes + Q * pop_bytes);
        for (int j = j0, x = x0; j < tl.y;) {
            {
                if (j != rj) {
                    rj = j;
                    rr = row_refs<T>(v, y0 + j, z0, PARITY == 1);
                }
                const int L = j * nx + x;
                const int xm = (x == 0 ? nx : x) - 1, xp = (x == nx - 1 ? -1 : x) + 1;
                // the value arriving from direction i sits in direction i's
                // range at x - c_i on odd steps (x wrapped), at x on even
                // steps; the range offsets i * TNM are constants
                T *const b0 = P + L, *const bm = P + (j * nx + xm), *const bp = P + (j * nx + xp);
                auto at = [&](int i) -> T & {
                    return (PARITY == 0 ? b0 : (cx(i) > 0 ? bm : (cx(i) < 0 ? bp : b0)))[i * TNM];
                };
                R d[Q], p[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    d[i] = dec<T, R>(at(i), PARITY ? ref_dir(i, rr.at(-cy(i), -cz(i))) : ref_dir(i, rr.own),
                                     cx(i) != 0);
                R rho, ux, uy, uz;
                const R om = (v.ind && v.ind[(size_t)tl.x * nx + L]) ? v.omega_in : v.omega;
                bgk_guo<R>(d, Fs[L], Fs[TNM + L], Fs[2 * TNM + L], om, p, rho, ux, uy, uz);
                if (v.rec) {
                    const size_t n = (size_t)tl.x * nx + L;
                    v.rec[n] = rho;
                    v.rec[N + n] = ux;
                    v.rec[2 * N + n] = uy;
                    v.rec[3 * N + n] = uz;
                }
                // outgoing direction i takes the place of incoming opp(i)
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    at(opp(i)) = enc<T, R>(p[i], PARITY ? ref_dir(i, rr.at(cy(i), cz(i))) : ref_dir(i, rr.own));
            }
            x += dx;
            j += dj;
            if (x >= nx) {
                x -= nx;
                ++j;
            }
        }
        tl = tl_next;
        fence_async_smem();  // this thread's writes, before the producer's bulk stores read them
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
    }
}

// The rows next to walls of a staging plan, node by node, one node per
// thread: their nodes own population slots disjoint from the tiles', so
// the order of the two kernels does not matter.
template <typename T, typename R, int PARITY, typename I>
__global__ void __launch_bounds__(256, 4) collide_erows_kernel(View<R> v) {
    const int nx = v.nx;
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    if (t >= (long long)v.nerows * nx) return;
    const int jr = (int)(t / nx);
    collide_node<T, R, PARITY, I>(v, v.erows[jr] * nx + (int)(t - (long long)jr * nx));
}

// post-streaming velocity u = (sum f c + F/2) / rho with the force just
// applied; LAYOUT as in load_pops.  Flags non-finite or |u| > 0.3.
template <typename T, typename R, int LAYOUT, bool LINKS, typename I>
__device__ __forceinline__ void moments_core(const View<R> &v, int n, const Nbr &o, uint64_t lk, const RowRefs &rr) {
    R d[Q];
    load_pops<T, R, LAYOUT, LINKS, I>(v, n, lk, o, rr, d);
    R drho = R(0), mx = R(0), my = R(0), mz = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += d[i];
        if (cx(i)) mx += cx(i) > 0 ? d[i] : -d[i];
        if (cy(i)) my += cy(i) > 0 ? d[i] : -d[i];
        if (cz(i)) mz += cz(i) > 0 ? d[i] : -d[i];
    }
    const size_t N = (size_t)v.N;
    const R inv = recip(R(1) + drho);
    const R ux = (mx + R(0.5) * v.F[n]) * inv;
    const R uy = (my + R(0.5) * v.F[N + n]) * inv;
    const R uz = (mz + R(0.5) * v.F[2 * N + n]) * inv;
    v.u[n] = ux;
    v.u[N + n] = uy;
    v.u[2 * N + n] = uz;
    const float q = (float)(ux * ux + uy * uy + uz * uz);
    if (!(q < U_LIMIT2)) atomicOr(v.status, ST_NUMERIC);
}

template <typename T, typename R, int LAYOUT, typename I>
__global__ void __launch_bounds__(NODE_BX * MOM_BY) moments_kernel(View<R> v) {
    const int x = blockIdx.x * NODE_BX + threadIdx.x, y = blockIdx.y * MOM_BY + threadIdx.y, z = blockIdx.z;
    if (x >= v.nx || y >= v.ny) return;
    const int n = x + v.nx * (y + v.ny * z);
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
    const RowRefs rr = row_refs<T>(v, y, z, LAYOUT == 1);
    if (nt & 0x80) moments_core<T, R, LAYOUT, true, I>(v, n, nbr_at(v, x, y, z), v.links[n], rr);
    else moments_core<T, R, LAYOUT, false, I>(v, n, nbr_at(v, x, y, z), 0ull, rr);
}

// ---------------------------------------------------------------------------
// 16-bit storage, two nodes per thread.
//
// With 2-byte populations a thread that collides one node keeps 38 bytes of
// loads in flight, too few to cover the memory latency at the occupancy the
// collision allows.  Here lane L of a warp takes the nodes x0 = 64 b + 2 L
// and x0 + 1 of one row (b the warp's chunk of the row; nx even, so that the
// pair is one aligned 32-bit word of every direction's range): 19 loads and
// 19 stores of 4 bytes for the two nodes.  Where a direction's reads or
// writes are one node off the pair (cx_i != 0 on odd steps, and for the
// velocity after an even step), a lane takes its own aligned word and the
// neighbouring lane's by a warp shuffle; the first and the last lane of a
// chunk fetch or store the one value that lies in the neighbouring chunk
// with a 2-byte access (x wrapped at the row's ends).  A warp whose nodes
// are not all fluid without wall links collides them one by one
// (collide_at).  The arithmetic per node is the per-node kernel's, so the
// results are the same bits.
// ---------------------------------------------------------------------------
template <typename T> struct Bits;
template <> struct Bits<__half> {
    static __device__ __forceinline__ __half of(unsigned short b) { return __ushort_as_half(b); }
    static __device__ __forceinline__ unsigned short to(__half h) { return __half_as_ushort(h); }
};
template <> struct Bits<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 of(unsigned short b) { return __ushort_as_bfloat16(b); }
    static __device__ __forceinline__ unsigned short to(__nv_bfloat16 h) { return __bfloat16_as_ushort(h); }
};
// the low / high 16-bit value of a pair word, decoded with reference ref
// (not added when has_ref is false, as in dec)
template <typename T> __device__ __forceinline__ float dec_lo(unsigned w, float ref, bool has_ref) {
    const float x = Store<T>::ld(Bits<T>::of((unsigned short)(w & 0xffffu)));
    return has_ref ? x + ref : x;
}
template <typename T> __device__ __forceinline__ float dec_hi(unsigned w, float ref, bool has_ref) {
    const float x = Store<T>::ld(Bits<T>::of((unsigned short)(w >> 16)));
    return has_ref ? x + ref : x;
}
template <typename T> __device__ __forceinline__ unsigned enc16(float q, float ref) {
    return Bits<T>::to(Store<T>::st(q - ref));
}
template <typename T> __device__ __forceinline__ unsigned ld_pair(const T *p) { return *reinterpret_cast<const unsigned *>(p); }
template <typename T> __device__ __forceinline__ unsigned ld_one(const T *p) { return Bits<T>::to(*p); }
template <typename T> __device__ __forceinline__ void st_pair(T *p, unsigned w) { *reinterpret_cast<unsigned *>(p) = w; }
template <typename T> __device__ __forceinline__ void st_one(T *p, unsigned b) { *p = Bits<T>::of((unsigned short)b); }

constexpr int PAIR_X = 2 * NODE_BX;  // nodes of a row per warp

// The 19 pair words arriving at nodes x0, x0 + 1 (low half: node x0).
// LAYOUT 0: natural order; 1: after an even step (direction i from slot
// opp(i) of the nodes x - c_i).  Where that is one node off the pair
// (cx_i != 0), the two aligned words around it are loaded and the halves
// picked, so that every load is independent and all are in flight at once.
// row0: index of the row's node x = 0; o: the row's y and z neighbour
// offsets; xb2, xa2: the pair positions before and after x0 (wrapped).
template <typename T, int LAYOUT, typename I>
__device__ __forceinline__ void load_pair_words(const View<float> &v, int n0, int row0, int xb2, int xa2, const Nbr &o,
                                                bool act, unsigned w[Q]) {
    const T *f = (const T *)v.f;
    const I N = (I)v.N;
    unsigned e[Q];  // the second word of the directions read one node off
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int roff = LAYOUT == 0 ? 0 : o.of(0, -cy(i), -cz(i));
        const T *src = f + (I)(LAYOUT == 0 ? i : opp(i)) * N;
        w[i] = act ? ld_pair(src + (I)(n0 + roff)) : 0u;  // values at x0, x0 + 1
        if (LAYOUT == 1 && cx(i) != 0)  // values at x0 - 2, x0 - 1 or x0 + 2, x0 + 3
            e[i] = act ? ld_pair(src + (I)(row0 + roff + (cx(i) > 0 ? xb2 : xa2))) : 0u;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (LAYOUT == 1 && cx(i) > 0) w[i] = (e[i] >> 16) | (w[i] << 16);          // from x0 - 1, x0
        else if (LAYOUT == 1 && cx(i) < 0) w[i] = (w[i] >> 16) | (e[i] << 16);     // from x0 + 1, x0 + 2
    }
}

template <typename T, int PARITY, typename I, bool VISC>
__global__ void __launch_bounds__(NODE_BX * NODE_BY) collide_pair_kernel(View<float> v) {
    drop_dead_lines(v);
    const int lane = threadIdx.x;
    const int x0 = blockIdx.x * PAIR_X + 2 * lane, y = blockIdx.y * NODE_BY + threadIdx.y, z = blockIdx.z;
    if (y >= v.ny) return;  // the whole warp (threadIdx.y is uniform in a warp)
    const int nx = v.nx;
    const bool act = x0 < nx;
    const int row0 = nx * (y + v.ny * z), n0 = row0 + x0;
    const uint8_t t0 = act ? v.ntype[n0] : 0, t1 = act ? v.ntype[n0 + 1] : 0;
    if (!__all_sync(0xffffffffu, (t0 | t1) == 0)) {  // walls or wall links in this chunk
        if (act) {
            collide_at<T, float, PARITY, I, VISC>(v, n0, x0, y, z);
            collide_at<T, float, PARITY, I, VISC>(v, n0 + 1, x0 + 1, y, z);
        }
        return;
    }
    const bool first = lane == 0, last = lane == 31 || x0 + 2 >= nx;
    const int xb = x0 == 0 ? nx - 1 : x0 - 1, xa = x0 + 2 >= nx ? 0 : x0 + 2;
    const Nbr o = nbr_at(v, x0, y, z);
    const RowRefs rr = row_refs<T>(v, y, z, PARITY == 1);
    unsigned w[Q];
    load_pair_words<T, PARITY, I>(v, n0, row0, x0 == 0 ? nx - 2 : x0 - 2, xa, o, act, w);
    const size_t N = (size_t)v.N;
    const float2 F0 = act ? *reinterpret_cast<const float2 *>(v.F + n0) : make_float2(0.f, 0.f);
    const float2 F1 = act ? *reinterpret_cast<const float2 *>(v.F + N + n0) : make_float2(0.f, 0.f);
    const float2 F2 = act ? *reinterpret_cast<const float2 *>(v.F + 2 * N + n0) : make_float2(0.f, 0.f);
    // reference of direction i as read and as written (the slots' rows)
    auto ref_rd = [&](int i) { return PARITY == 0 ? ref_dir(i, rr.own) : ref_dir(i, rr.at(-cy(i), -cz(i))); };
    auto ref_wr = [&](int i) { return PARITY == 0 ? ref_dir(i, rr.own) : ref_dir(i, rr.at(cy(i), cz(i))); };
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // node x0 (low halves), then x0 + 1 (high halves)
        const int n = n0 + h;
        float d[Q], p[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            d[i] = h ? dec_hi<T>(w[i], ref_rd(i), cx(i) != 0) : dec_lo<T>(w[i], ref_rd(i), cx(i) != 0);
        const float om = (VISC && act && v.ind && v.ind[n]) ? v.omega_in : v.omega;
        float rho, ux, uy, uz;
        bgk_guo<float>(d, h ? F0.y : F0.x, h ? F1.y : F1.x, h ? F2.y : F2.x, om, p, rho, ux, uy, uz);
        if (v.rec && act) {
            v.rec[n] = rho;
            v.rec[N + n] = ux;
            v.rec[2 * N + n] = uy;
            v.rec[3 * N + n] = uz;
        }
        // the outputs replace this node's half of the words (the other
        // node's inputs stay in the other half)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const unsigned e = enc16<T>(p[i], ref_wr(i));
            w[i] = h ? ((w[i] & 0xffffu) | (e << 16)) : ((w[i] & 0xffff0000u) | e);
        }
    }
    T *f = (T *)v.f;
    const I NI = (I)N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (PARITY == 0) {  // direction i leaving x0, x0 + 1: slot opp(i)
            if (act) st_pair(f + (I)opp(i) * NI + (I)n0, w[i]);
        } else {  // direction i arriving at x + c_i: slot i
            const int roff = o.of(0, cy(i), cz(i));
            T *dst = f + (I)i * NI;
            if (cx(i) == 0) {
                if (act) st_pair(dst + (I)(n0 + roff), w[i]);
            } else if (cx(i) > 0) {  // x0 -> x0 + 1, x0 + 1 -> x0 + 2
                const unsigned left = __shfl_up_sync(0xffffffffu, w[i], 1);
                if (act) {
                    if (first) st_one(dst + (I)(n0 + roff + 1), w[i] & 0xffffu);
                    else st_pair(dst + (I)(n0 + roff), (left >> 16) | (w[i] << 16));
                    if (last) st_one(dst + (I)(row0 + roff + xa), w[i] >> 16);
                }
            } else {  // x0 -> x0 - 1, x0 + 1 -> x0
                const unsigned right = __shfl_down_sync(0xffffffffu, w[i], 1);
                if (act) {
                    if (last) st_one(dst + (I)(n0 + roff), w[i] >> 16);
                    else st_pair(dst + (I)(n0 + roff), (w[i] >> 16) | (right << 16));
                    if (first) st_one(dst + (I)(row0 + roff + xb), w[i] & 0xffffu);
                }
            }
        }
    }
}

// post-streaming velocity of two nodes per thread (16-bit storage); LAYOUT
// as in load_pops
template <typename T, int LAYOUT, typename I>
__global__ void __launch_bounds__(NODE_BX * MOM_BY) moments_pair_kernel(View<float> v) {
    const int lane = threadIdx.x;
    const int x0 = blockIdx.x * PAIR_X + 2 * lane, y = blockIdx.y * MOM_BY + threadIdx.y, z = blockIdx.z;
    if (y >= v.ny) return;
    const int nx = v.nx;
    const bool act = x0 < nx;
    const int row0 = nx * (y + v.ny * z), n0 = row0 + x0;
    const uint8_t t0 = act ? v.ntype[n0] : 0, t1 = act ? v.ntype[n0 + 1] : 0;
    if (!__all_sync(0xffffffffu, (t0 | t1) == 0)) {
        if (act)
            for (int h = 0; h < 2; ++h) {
                const int n = n0 + h;
                const uint8_t nt = h ? t1 : t0;
                if (nt & 0x7f) {  // wall node: the wall's velocity (written when recording into a fresh buffer)
                    if (v.rec)
                        for (int k = 0; k < 3; ++k) v.u[(size_t)k * v.N + n] = v.uw[nt & 0x7f][k];
                    continue;
                }
                const Nbr o = nbr_at(v, x0 + h, y, z);
                const RowRefs rr = row_refs<T>(v, y, z, LAYOUT == 1);
                if (nt & 0x80) moments_core<T, float, LAYOUT, true, I>(v, n, o, v.links[n], rr);
                else moments_core<T, float, LAYOUT, false, I>(v, n, o, 0ull, rr);
            }
        return;
    }
    const int xa = x0 + 2 >= nx ? 0 : x0 + 2;
    const Nbr o = nbr_at(v, x0, y, z);
    const RowRefs rr = row_refs<T>(v, y, z, LAYOUT == 1);
    unsigned w[Q];
    load_pair_words<T, LAYOUT, I>(v, n0, row0, x0 == 0 ? nx - 2 : x0 - 2, xa, o, act, w);
    if (!act) return;
    const size_t N = (size_t)v.N;
    float u[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float drho = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float ref = LAYOUT == 0 ? ref_dir(i, rr.own) : ref_dir(i, rr.at(-cy(i), -cz(i)));
            const float d = h ? dec_hi<T>(w[i], ref, cx(i) != 0) : dec_lo<T>(w[i], ref, cx(i) != 0);
            drho += d;
            if (cx(i)) mx += cx(i) > 0 ? d : -d;
            if (cy(i)) my += cy(i) > 0 ? d : -d;
            if (cz(i)) mz += cz(i) > 0 ? d : -d;
        }
        const int n = n0 + h;
        const float inv = recip(1.f + drho);
        u[h][0] = (mx + 0.5f * v.F[n]) * inv;
        u[h][1] = (my + 0.5f * v.F[N + n]) * inv;
        u[h][2] = (mz + 0.5f * v.F[2 * N + n]) * inv;
        const float q = u[h][0] * u[h][0] + u[h][1] * u[h][1] + u[h][2] * u[h][2];
        if (!(q < U_LIMIT2)) atomicOr(v.status, ST_NUMERIC);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) *reinterpret_cast<float2 *>(v.u + k * N + n0) = make_float2(u[0][k], u[1][k]);
}

// Rows' reference x-velocity from a velocity field u0 ([n][3], double):
// the mean of u_x over the row's fluid nodes (0 for a row without fluid),
// stored as (P, M) (see row_refs)
__global__ void row_reference_kernel(int nx, int nrows, const uint8_t *ntype, const double *u0, float2 *rref) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    double s = 0;
    int k = 0;
    for (int x = 0; x < nx; ++x) {
        const size_t n = (size_t)r * nx + x;
        if (ntype[n] & 0x7f) continue;
        s += u0[3 * n];
        ++k;
    }
    const double U = k ? s / k : 0.0;
    rref[r] = make_float2((float)((3.0 * U + 3.0 * U * U) / 18.0), (float)((-3.0 * U + 3.0 * U * U) / 18.0));
}

// Natural-order 16-bit populations re-stored from reference table `from` to
// table `to` (either may be null: zero reference)
template <typename T>
__global__ void reencode_kernel(View<float> v, const float2 *from, const float2 *to) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= v.N) return;
    if (v.ntype[n] & 0x7f) return;
    const int r = n / v.nx;
    const float2 a = from ? from[r] : make_float2(0.f, 0.f), b = to ? to[r] : make_float2(0.f, 0.f);
    T *f = (T *)v.f;
    const size_t N = (size_t)v.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T &s = f[(size_t)i * N + n];
        s = Store<T>::st(Store<T>::ld(s) + ref_dir(i, a) - ref_dir(i, b));
    }
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
    const RowRefs rr = row_refs_of<T>(v, n, false);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        f[(size_t)i * N + n] = enc<T, R>(R(wgt(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu)), ref_dir(i, rr.own));
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
    load_pops<T, R, LAYOUT, true>(v, n, lk, nb, row_refs_of<T>(v, n, LAYOUT == 1), d);
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
    load_pops<T, R, LAYOUT, true>(v, n, lk, nb, row_refs_of<T>(v, n, LAYOUT == 1), d);
    R drho = R(0);
    for (int i = 0; i < Q; ++i) drho += d[i];
    out[n] = R(1) + drho;
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
    load_pops<T, R, LAYOUT, true>(v, n, lk, o, row_refs_of<T>(v, n, LAYOUT == 1), d);
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
    const RowRefs rr = row_refs_of<T>(v, n, LAYOUT == 1);
    for (int i = 0; i < Q; ++i) {  // the slot and its reference as load_pops reads them
        const R val = in[(size_t)i * N + n];
        if (LAYOUT == 0) f[(size_t)i * N + n] = enc<T, R>(val, ref_dir(i, rr.own));
        else if (i == 0) f[n] = enc<T, R>(val, 0.f);
        else if (link_code(lk, opp(i))) f[(size_t)i * N + n] = enc<T, R>(val, ref_dir(opp(i), rr.own));
        else f[(size_t)opp(i) * N + n + o.of(-cx(i), -cy(i), -cz(i))] = enc<T, R>(val, ref_dir(i, rr.at(-cy(i), -cz(i))));
    }
}

inline int nblocks(long long n, int b) { return (int)((n + b - 1) / b); }
// 32-bit population indices when every index i N + n fits (unless 64-bit
// ones are asked for)
template <typename R>
bool narrow_index(const View<R> &v) {
    return !v.wide_index && (unsigned long long)Q * (unsigned long long)v.N <= 0xffffffffull;
}
template <typename R>
dim3 node_grid(const View<R> &v) {
    return dim3((unsigned)nblocks(v.nx, NODE_BX), (unsigned)nblocks(v.ny, NODE_BY), (unsigned)v.nz);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

// the per-node kernel, or for 16-bit storage the two-node kernel
template <typename T, typename R, int PARITY, typename I, bool VISC>
void launch_collide_as(const View<R> &v, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value && sizeof(T) == 2) {
        if (v.node_pairs & PAIR_COLLIDE) {
            const dim3 g((unsigned)nblocks(v.nx, PAIR_X), (unsigned)nblocks(v.ny, NODE_BY), (unsigned)v.nz);
            collide_pair_kernel<T, PARITY, I, VISC><<<g, dim3(NODE_BX, NODE_BY), 0, st>>>(v);
            return;
        }
    }
    collide_stream_kernel<T, R, PARITY, I, VISC><<<node_grid(v), dim3(NODE_BX, NODE_BY), 0, st>>>(v);
}

template <typename T, typename R, typename I>
void launch_collide_parity(const View<R> &v, int parity, cudaStream_t st) {
    const bool visc = v.ind != nullptr;  // internal viscosity on
    if (parity == 0) {
        if (visc) launch_collide_as<T, R, 0, I, true>(v, st);
        else launch_collide_as<T, R, 0, I, false>(v, st);
    } else {
        if (visc) launch_collide_as<T, R, 1, I, true>(v, st);
        else launch_collide_as<T, R, 1, I, false>(v, st);
    }
}

template <typename T, typename R, int PARITY, typename I>
void launch_tiles_pi(const View<R> &v, cudaStream_t st) {
    collide_tiles_kernel<T, R, PARITY, I><<<v.tile_grid, TILE_THREADS, v.tile_smem, st>>>(v);
    const long long ne = (long long)v.nerows * v.nx;
    if (ne > 0) collide_erows_kernel<T, R, PARITY, I><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(v);
}

template <typename T, typename R>
void launch_tiles_as(const View<R> &v, int parity, cudaStream_t st) {
    if (narrow_index(v)) {
        if (parity) launch_tiles_pi<T, R, 1, unsigned>(v, st);
        else launch_tiles_pi<T, R, 0, unsigned>(v, st);
    } else {
        if (parity) launch_tiles_pi<T, R, 1, size_t>(v, st);
        else launch_tiles_pi<T, R, 0, size_t>(v, st);
    }
}

template <typename R>
void launch_collide(const View<R> &v, int precision, int parity, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value) {
        // 16-bit storage with a staging plan: the staged kernel, which also
        // collides the rows next to walls node by node once its tiles are done
        if (v.ntiles && (precision == HEMO_F16DEV || precision == HEMO_BF16DEV)) {
            if (precision == HEMO_F16DEV) launch_tiles_as<__half, R>(v, parity, st);
            else launch_tiles_as<__nv_bfloat16, R>(v, parity, st);
            return;
        }
    }
    if (narrow_index(v)) HEMO_DISPATCH_T(precision, R, (launch_collide_parity<T, R, unsigned>(v, parity, st)));
    else HEMO_DISPATCH_T(precision, R, (launch_collide_parity<T, R, size_t>(v, parity, st)));
}

cudaError_t set_tile_smem_limit(int precision, int bytes) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    auto set_all = [&](auto tag) {
        using T = decltype(tag);
        set((const void *)collide_tiles_kernel<T, float, 1, unsigned>);
        set((const void *)collide_tiles_kernel<T, float, 1, size_t>);
        set((const void *)collide_tiles_kernel<T, float, 0, unsigned>);
        set((const void *)collide_tiles_kernel<T, float, 0, size_t>);
    };
    if (precision == HEMO_F16DEV) set_all(__half());
    else if (precision == HEMO_BF16DEV) set_all(__nv_bfloat16());
    return e;
}


template <typename T, typename R, int LAYOUT, typename I>
void launch_moments_as(const View<R> &v, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value && sizeof(T) == 2) {
        if (v.node_pairs & PAIR_MOMENTS) {
            const dim3 g((unsigned)nblocks(v.nx, PAIR_X), (unsigned)nblocks(v.ny, MOM_BY), (unsigned)v.nz);
            moments_pair_kernel<T, LAYOUT, I><<<g, dim3(NODE_BX, MOM_BY), 0, st>>>(v);
            return;
        }
    }
    const dim3 g((unsigned)nblocks(v.nx, NODE_BX), (unsigned)nblocks(v.ny, MOM_BY), (unsigned)v.nz);
    moments_kernel<T, R, LAYOUT, I><<<g, dim3(NODE_BX, MOM_BY), 0, st>>>(v);
}

template <typename R>
void launch_moments(const View<R> &v, int precision, int parity, cudaStream_t st) {
    // after an even step the array is in the swapped layout (1), after an odd
    // step in natural order (0)
    if (narrow_index(v)) {
        if (parity == 0) HEMO_DISPATCH_T(precision, R, (launch_moments_as<T, R, 1, unsigned>(v, st)));
        else HEMO_DISPATCH_T(precision, R, (launch_moments_as<T, R, 0, unsigned>(v, st)));
    } else {
        if (parity == 0) HEMO_DISPATCH_T(precision, R, (launch_moments_as<T, R, 1, size_t>(v, st)));
        else HEMO_DISPATCH_T(precision, R, (launch_moments_as<T, R, 0, size_t>(v, st)));
    }
}

void launch_row_reference(const View<float> &v, const double *u0, float2 *rref, cudaStream_t st) {
    const int nrows = v.ny * v.nz;
    row_reference_kernel<<<nblocks(nrows, 128), 128, 0, st>>>(v.nx, nrows, v.ntype, u0, rref);
}

void launch_reencode(const View<float> &v, int precision, const float2 *from, const float2 *to, cudaStream_t st) {
    if (precision == HEMO_F16DEV) reencode_kernel<__half><<<nblocks(v.N, 256), 256, 0, st>>>(v, from, to);
    else if (precision == HEMO_BF16DEV) reencode_kernel<__nv_bfloat16><<<nblocks(v.N, 256), 256, 0, st>>>(v, from, to);
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
