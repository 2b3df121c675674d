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

#include "lattice_core.cuh"

namespace hemo {

namespace {

// Read the 19 populations arriving at node n.  LAYOUT 0: natural order (slot
// i of n).  LAYOUT 1: after an even step (slot opp(i) of n - c_i, or slot i
// of n when n - c_i is a wall).  LINKS false: no wall among the neighbours
// (lk is not read).  I: the index type of the population array, 32-bit
// unsigned when 19 N < 2^32 (fewer registers and address instructions).
template <typename T, typename R, int LAYOUT, bool LINKS, typename I = size_t>
__device__ __forceinline__ void load_pops(const View<R> &v, int n, uint64_t lk, const Nbr &o, R d[Q]) {
    const T *f = (const T *)v.f;
    const I N = (I)v.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (LAYOUT == 0) {
            d[i] = Store<T>::ld(f[(I)i * N + (I)n]);
        } else {
            if (i == 0) {
                d[i] = Store<T>::ld(f[n]);
            } else if (LINKS && link_code(lk, opp(i))) {
                d[i] = Store<T>::ld(f[(I)i * N + (I)n]);
            } else {
                d[i] = Store<T>::ld(f[(I)opp(i) * N + (I)(n + o.of(-cx(i), -cy(i), -cz(i)))]);
            }
        }
    }
}

// collision and streaming of fluid node n with neighbour offsets o,
// reading and writing the global array directly; LINKS false for a node
// without wall neighbours (most of them: that path carries no wall terms)
template <typename T, typename R, int PARITY, bool LINKS, typename I, bool VISC = true>
__device__ __forceinline__ void collide_core(const View<R> &v, int n, const Nbr &o, uint64_t lk) {
    R d[Q], p[Q];
    load_pops<T, R, PARITY, LINKS, I>(v, n, lk, o, d);
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
        if (PARITY == 0) {
            f[(I)opp(i) * NI + (I)n] = Store<T>::st(q);
        } else {
            if (code)
                f[(I)opp(i) * NI + (I)n] = Store<T>::st(q);
            else
                f[(I)i * NI + (I)(n + o.of(cx(i), cy(i), cz(i)))] = Store<T>::st(q);
        }
    }
}

// node (x, y, z) = index n; VISC: the internal viscosity may be on
template <typename T, typename R, int PARITY, typename I, bool VISC>
__device__ __forceinline__ void collide_at(const View<R> &v, int n, int x, int y, int z) {
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) return;  // wall node
    if (nt & 0x80) collide_core<T, R, PARITY, true, I, VISC>(v, n, nbr_at(v, x, y, z), v.links[n]);
    else collide_core<T, R, PARITY, false, I, VISC>(v, n, nbr_at(v, x, y, z), 0ull);
}

// any node given by its index (walls included), one code path for nodes
// with and without wall links (the rows next to walls)
template <typename T, typename R, int PARITY, typename I>
__device__ __forceinline__ void collide_node(const View<R> &v, int n) {
    const uint8_t nt = v.ntype[n];
    if (nt & 0x7f) return;  // wall node
    const int r = n / v.nx;
    collide_core<T, R, PARITY, true, I>(v, n, nbr_at(v, n % v.nx, r % v.ny, r / v.ny), (nt & 0x80) ? v.links[n] : 0ull);
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
// x-shift applied in shared memory with the periodic wrap).  A persistent CTA
// copies them, with the force rows, into a ring of shared-memory stages by
// bulk copies (cp.async.bulk, completion on an mbarrier), collides in place
// (each node writes its outgoing value where the opposite incoming value was)
// and writes the same ranges back by bulk stores; the CTAs then collide the
// rows next to walls node by node.  The ring keeps several
// tiles of loads in flight per SM without holding them in registers, which
// is what 2-byte populations need to reach the HBM bandwidth; four CTAs of
// 256 threads share an SM, so that one computes while another waits.
constexpr int TILE_THREADS = 256;
constexpr int TILE_CTAS_PER_SM = 4;
constexpr int TILE_NODES = 256;  // stride of a direction's range in a stage (nodes)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// waits for the phase with the given parity; gives up after about a second
__device__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 256; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
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

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// The rows of a tile (k rows from global row r0 = y0 + ny z) shifted by
// (dy, dz), as at most two contiguous pieces (a periodic wrap in y splits
// them): fn(first element of the piece in the lattice, first element in the
// tile buffer, element count).
template <typename R, typename Fn>
__device__ __forceinline__ void tile_pieces(const View<R> &v, int r0, int k, int dy, int dz, Fn fn) {
    const int y0 = r0 % v.ny, z = r0 / v.ny;
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

constexpr int TILE_COPIES = Q + 3;  // lanes of warp 0 that issue the copies of a stage

template <typename T, typename R, int PARITY, typename I>
__global__ void __launch_bounds__(TILE_THREADS, TILE_CTAS_PER_SM) collide_tiles_kernel(View<R> v) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *ring = smem + 128;
    constexpr int TNM = TILE_NODES;
    constexpr size_t pop_bytes = (size_t)TNM * sizeof(T), stage_bytes = Q * pop_bytes + 3 * (size_t)TNM * sizeof(R);
    const int nx = v.nx, S = v.tile_stages;
    const size_t N = (size_t)v.N;
    const int ntiles = v.ntiles;
    const int lane = threadIdx.x;  // meaningful in warp 0
    const bool issuer = threadIdx.x < TILE_COPIES, storer = threadIdx.x < Q;
    auto tile_of = [&](int it) { return (int)blockIdx.x + it * (int)gridDim.x; };
    T *f = (T *)v.f;

    // Lane i < 19 of warp 0 copies direction i's range (slot i of the tile's
    // rows on even steps, slot opp(i) of the rows shifted by -c_i on odd
    // steps); lanes 19..21 copy the three force components.  Each lane
    // announces its own bytes on the stage's barrier (22 arrivals).
    auto issue_load = [&](int it) {
        const int2 tl = v.rtiles[tile_of(it)];
        const int s = it % S;
        unsigned char *st = ring + s * stage_bytes;
        const unsigned tn = (unsigned)(tl.y * nx);
        if (lane < Q) {
            T *buf = (T *)(st + lane * pop_bytes);
            const T *src = f + (size_t)(PARITY ? opp(lane) : lane) * N;
            mbar_expect_tx(bar + s, tn * (unsigned)sizeof(T));
            tile_pieces(v, tl.x, tl.y, PARITY ? -cy_of(lane) : 0, PARITY ? -cz_of(lane) : 0,
                        [&](long long g, int b, int cnt) {
                            bulk_load(buf + b, src + g, (unsigned)(cnt * sizeof(T)), bar + s);
                        });
        } else {
            const int c = lane - Q;
            R *fs = (R *)(st + Q * pop_bytes) + c * TNM;
            mbar_expect_tx(bar + s, tn * (unsigned)sizeof(R));
            bulk_load(fs, v.F + c * N + (size_t)tl.x * nx, tn * (unsigned)sizeof(R), bar + s);
        }
    };
    auto issue_store = [&](int it) {  // lane < 19: the range it loaded
        const int2 tl = v.rtiles[tile_of(it)];
        unsigned char *st = ring + (it % S) * stage_bytes;
        T *buf = (T *)(st + lane * pop_bytes);
        T *dst = f + (size_t)(PARITY ? opp(lane) : lane) * N;
        tile_pieces(v, tl.x, tl.y, PARITY ? -cy_of(lane) : 0, PARITY ? -cz_of(lane) : 0,
                    [&](long long g, int b, int cnt) { bulk_store(dst + g, buf + b, (unsigned)(cnt * sizeof(T))); });
        bulk_commit();
    };

    drop_dead_lines(v);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) mbar_init(bar + s, TILE_COPIES);
        fence_mbar_init();
    }
    __syncthreads();
    if (issuer)
        for (int it = 0; it < S - 1 && tile_of(it) < ntiles; ++it) issue_load(it);

    for (int it = 0; tile_of(it) < ntiles; ++it) {
        const int s = it % S;
        const bool ok = mbar_wait(bar + s, (unsigned)((it / S) & 1));
        if (__syncthreads_or(!ok)) {  // let the copies in flight land, then report
            if (threadIdx.x == 0)
                for (int j = it; j < it + S - 1 && tile_of(j) < ntiles; ++j)
                    mbar_wait(bar + j % S, (unsigned)((j / S) & 1));
            if (storer) bulk_wait_read<0>();
            if (threadIdx.x == 0) atomicOr(v.status, ST_TIMEOUT);
            return;
        }
        const int2 tl = v.rtiles[tile_of(it)];
        const int TN = tl.y * nx;
        T *P = (T *)(ring + s * stage_bytes);
        const R *Fs = (const R *)(ring + s * stage_bytes + Q * pop_bytes);
        for (int L = threadIdx.x; L < TN; L += TILE_THREADS) {
            const int j = L / nx, x = L - j * nx;
            const int xm = (x == 0 ? nx : x) - 1, xp = (x == nx - 1 ? -1 : x) + 1;
            // the value arriving from direction i sits in direction i's range
            // at x - c_i on odd steps (x wrapped), at x on even steps; the
            // range offsets i * TNM are constants
            T *const b0 = P + L, *const bm = P + (j * nx + xm), *const bp = P + (j * nx + xp);
            auto at = [&](int i) -> T & {
                return (PARITY == 0 ? b0 : (cx(i) > 0 ? bm : (cx(i) < 0 ? bp : b0)))[i * TNM];
            };
            R d[Q], p[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) d[i] = Store<T>::ld(at(i));
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
            for (int i = 0; i < Q; ++i) at(opp(i)) = Store<T>::st(p[i]);
        }
        fence_async_smem();
        __syncthreads();
        if (storer) issue_store(it);
        if (issuer && tile_of(it + S - 1) < ntiles) {
            if (storer) bulk_wait_read<1>();  // this lane's range of tile it - 1 has been written out
            issue_load(it + S - 1);           // into the stage tile it - 1 used
        }
    }
    if (storer) bulk_wait_read<0>();
    // then the rows next to walls, node by node: their nodes own population
    // slots disjoint from the tiles', so the order does not matter
    const long long ne = (long long)v.nerows * nx;
    for (long long t = (long long)blockIdx.x * TILE_THREADS + threadIdx.x; t < ne; t += (long long)gridDim.x * TILE_THREADS) {
        const int jr = (int)(t / nx);
        collide_node<T, R, PARITY, I>(v, v.erows[jr] * nx + (int)(t - (long long)jr * nx));
    }
}

// post-streaming velocity u = (sum f c + F/2) / rho with the force just
// applied; LAYOUT as in load_pops.  Flags non-finite or |u| > 0.3.
template <typename T, typename R, int LAYOUT, bool LINKS, typename I>
__device__ __forceinline__ void moments_core(const View<R> &v, int n, const Nbr &o, uint64_t lk) {
    R d[Q];
    load_pops<T, R, LAYOUT, LINKS, I>(v, n, lk, o, d);
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
__global__ void __launch_bounds__(NODE_BX * NODE_BY) moments_kernel(View<R> v) {
    const int x = blockIdx.x * NODE_BX + threadIdx.x, y = blockIdx.y * NODE_BY + threadIdx.y, z = blockIdx.z;
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
    if (nt & 0x80) moments_core<T, R, LAYOUT, true, I>(v, n, nbr_at(v, x, y, z), v.links[n]);
    else moments_core<T, R, LAYOUT, false, I>(v, n, nbr_at(v, x, y, z), 0ull);
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
    load_pops<T, R, LAYOUT, true>(v, n, lk, nb, d);
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
    load_pops<T, R, LAYOUT, true>(v, n, lk, nb, d);
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
    load_pops<T, R, LAYOUT, true>(v, n, lk, o, d);
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
// 32-bit population indices when every index i N + n fits
template <typename R>
bool narrow_index(const View<R> &v) {
    return (unsigned long long)Q * (unsigned long long)v.N <= 0xffffffffull;
}
template <typename R>
dim3 node_grid(const View<R> &v) {
    return dim3((unsigned)nblocks(v.nx, NODE_BX), (unsigned)nblocks(v.ny, NODE_BY), (unsigned)v.nz);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <typename R>
void launch_collide(const View<R> &v, int precision, int parity, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value) {
        // 16-bit storage, odd steps (reads and writes shifted by one node in
        // x): the staged kernel, which also collides the rows next to walls
        // node by node once its tiles are done.  Even steps touch each node's
        // own slots, which the per-node kernel streams faster.
        if (v.ntiles && parity == 1) {
            if (narrow_index(v))
                HEMO_DISPATCH_T(precision, R, (collide_tiles_kernel<T, R, 1, unsigned><<<v.tile_grid, TILE_THREADS, v.tile_smem, st>>>(v)));
            else
                HEMO_DISPATCH_T(precision, R, (collide_tiles_kernel<T, R, 1, size_t><<<v.tile_grid, TILE_THREADS, v.tile_smem, st>>>(v)));
            return;
        }
    }
    const dim3 g = node_grid(v), b(NODE_BX, NODE_BY);
    if (v.ind) {  // internal viscosity on
        if (narrow_index(v)) {
            if (parity == 0)
                HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 0, unsigned, true><<<g, b, 0, st>>>(v)));
            else
                HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 1, unsigned, true><<<g, b, 0, st>>>(v)));
        } else {
            if (parity == 0)
                HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 0, size_t, true><<<g, b, 0, st>>>(v)));
            else
                HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 1, size_t, true><<<g, b, 0, st>>>(v)));
        }
    } else if (narrow_index(v)) {
        if (parity == 0)
            HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 0, unsigned, false><<<g, b, 0, st>>>(v)));
        else
            HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 1, unsigned, false><<<g, b, 0, st>>>(v)));
    } else {
        if (parity == 0)
            HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 0, size_t, false><<<g, b, 0, st>>>(v)));
        else
            HEMO_DISPATCH_T(precision, R, (collide_stream_kernel<T, R, 1, size_t, false><<<g, b, 0, st>>>(v)));
    }
}

cudaError_t set_tile_smem_limit(int precision, int bytes) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    using R = float;
    HEMO_DISPATCH_T(precision, R, (set((const void *)collide_tiles_kernel<T, R, 1, unsigned>)));
    HEMO_DISPATCH_T(precision, R, (set((const void *)collide_tiles_kernel<T, R, 1, size_t>)));
    return e;
}

template <typename R>
void launch_moments(const View<R> &v, int precision, int parity, cudaStream_t st) {
    // after an even step the array is in the swapped layout (1), after an odd
    // step in natural order (0)
    const dim3 g = node_grid(v), b(NODE_BX, NODE_BY);
    if (narrow_index(v)) {
        if (parity == 0)
            HEMO_DISPATCH_T(precision, R, (moments_kernel<T, R, 1, unsigned><<<g, b, 0, st>>>(v)));
        else
            HEMO_DISPATCH_T(precision, R, (moments_kernel<T, R, 0, unsigned><<<g, b, 0, st>>>(v)));
    } else {
        if (parity == 0)
            HEMO_DISPATCH_T(precision, R, (moments_kernel<T, R, 1, size_t><<<g, b, 0, st>>>(v)));
        else
            HEMO_DISPATCH_T(precision, R, (moments_kernel<T, R, 0, size_t><<<g, b, 0, st>>>(v)));
    }
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
