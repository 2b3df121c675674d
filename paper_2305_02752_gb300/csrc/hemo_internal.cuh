// Internal definitions shared by the CUDA translation units of libhemo.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hemo.h"

namespace hemo {

constexpr int Q = 19;
constexpr int BLK = 8;              // lattice block edge used for vertex bins
constexpr int MAX_TYPES = 8;        // membrane mesh types per simulation

// status bits raised on the device
constexpr unsigned ST_NUMERIC = 1u;
constexpr unsigned ST_DOMAIN = 2u;
constexpr unsigned ST_TIMEOUT = 4u;  // a pipeline wait gave up
constexpr unsigned ST_BOUNDS = 8u;   // an index failed its check (bounds-checked build only)

// The bounds-checked build (HEMO_BOUNDS_CHECK=1, libhemo_checked.so) tests
// the data-driven indices of the vertex, bin and membrane kernels (vertex
// ids read from the bin order, cell ids, mesh-table entries, bin slots)
// before use: a failed test sets ST_BOUNDS in the status word and the
// access is skipped.  In the default build index_ok is the constant true
// and the tests compile away.
#ifndef HEMO_BOUNDS_CHECK
#define HEMO_BOUNDS_CHECK 0
#endif
__device__ __forceinline__ bool index_ok(bool ok, unsigned *status) {
#if HEMO_BOUNDS_CHECK
    if (!ok && status) atomicOr(status, ST_BOUNDS);
    return ok;
#else
    (void)ok;
    (void)status;
    return true;
#endif
}
constexpr float U_LIMIT2 = 0.09f;   // |u|^2 above which the step is unstable
constexpr int PAIR_MOMENTS = 1, PAIR_COLLIDE = 2;  // View::node_pairs bits
constexpr int ADAPT_WORDS = 5;                      // View::adapt

// ---------------------------------------------------------------------------
// D3Q19 in the library's order: 0 rest; 1..6 = +x -x +y -y +z -z; 7..18 =
// diagonal pairs, each odd index followed by its opposite.  Weights 1/3,
// 1/18 (axis), 1/36 (diagonal); c_s^2 = 1/3 (Sec. 2.2).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) {
    constexpr int v[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[i];
}
__host__ __device__ constexpr int cy(int i) {
    constexpr int v[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[i];
}
__host__ __device__ constexpr int cz(int i) {
    constexpr int v[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// ---------------------------------------------------------------------------
// population storage: deviations d_i = f_i - w_i in T, arithmetic in R
// ---------------------------------------------------------------------------
template <typename T> struct Store;
template <> struct Store<double> {
    static __device__ __forceinline__ double ld(double v) { return v; }
    static __device__ __forceinline__ double st(double v) { return v; }
};
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(float v) { return v; }
    static __device__ __forceinline__ float st(float v) { return v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half st(float v) { return __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// device views (plain pointers, passed by value to kernels)
// ---------------------------------------------------------------------------
template <typename R> struct MeshDev {
    int nv, nt, ne;
    const int *tri;     // nt*3, in processing order
    const int *edge;    // ne*4: v0, v1, a, b, in processing order
    const int *etri;    // ne*2: the triangles (v0, v1, a) and (v1, v0, b), processing positions
    const R *invL0;     // ne: 1 / rest length
    const R *th0;       // ne: rest dihedral angle
    const int4 *tri4;   // nt: the triangle's corners, padded to 16 bytes
    int maxv;  // largest valence
    // per vertex its fan in cyclic order, slot-major (entry [slot * nv +
    // vertex]) over maxv + 1 slots, ids in processing order:
    // slot 0 = the last entry again, slots 1..deg the entries k = 0..deg-1,
    // then -1; entry {T_k, j_k, edge (i, j_k) << 1 | role, edge (j_k, j_k+1)}
    // with T_k = (i, j_k, j_k+1) as oriented
    const int4 *vfan;
    // strides coprime with nt and ne (about n/32): the FP64 adjoint takes
    // triangle and edge q * stride mod n, so that a warp's shared-memory
    // atomics fall on far-apart vertices
    int tstride, estride;
    // optional terms for large deformations (0 = off): per-triangle rest area
    // (processing order) and local area modulus; 1 / theta_m^2 of the
    // nonlinear bending term
    const R *At0;
    R k_local;
    R thm2i;
    double A0, V0;
    R K;                // k_link * kbt / persistence
    R m2;               // max_strain^2
    R kb;               // k_bend * kbt
    double k_area, k_volume;
    R Ku;               // kbt / persistence (link coefficient per unit k_link)
    R kbu;              // kbt (bending coefficient per unit k_bend)
    R k_link, k_bend;
};

template <typename R> struct View {
    // lattice
    int nx, ny, nz;
    long long N;
    int per[3];
    void *f;                   // 19*N deviations, storage type by precision
    const uint8_t *ntype;      // N: 0 fluid, 1..3 wall id, 0x80 = fluid next to a wall
    const uint64_t *links;     // N: 2 bits per direction (wall id of node + c_i)
    R *F;                      // [3][N] force density
    R *u;                      // [3][N] velocity
    R omega;
    R g[3];
    R uw[4][3];                // wall velocity by id
    // cells and vertices
    int nv, ncell;
    double *ctr;               // ncell*3 centroids (FP64)
    R *off;                    // nv*3 offsets from the centroid
    R *Fv;                     // nv*3 membrane forces
    const int *vcell;          // nv: cell of each vertex
    const int *cell_first;     // ncell
    const int *cell_type;      // ncell
    const MeshDev<R> *meshes;  // per type
    int max_nv;                // largest vertex count of a mesh type
    int max_nt;                // largest triangle count of a mesh type
    int max_ne;                // largest edge count of a mesh type
    int nsm;                   // multiprocessors of the device
    // bins
    int nb[3];
    int nbins;
    int *key;                  // nv
    int *counts;               // nbins
    int *start;                // nbins + 1
    int *cursor;               // nbins
    int *perm_raw;             // nv, unsorted within bins
    int *perm;                 // nv, stable (key, vertex id)
    int *anc_i;                // nv*3 stencil base floor(X) (wrapped on periodic axes)
    R *anc_t;                  // nv*3 fractions X - floor(X)
    R *tiles;                  // nbins*3*11^3 per-bin spreading tiles
    // vertex integrator (Sec. 2.6): 0 Euler X += U; 1 Euler and U kept in
    // Uprev; 2 Adams-Bashforth X += 3/2 U - 1/2 Uprev and U kept in Uprev
    int integ;
    R *Uprev;                  // nv*3 interpolated velocity of the previous step
    // adaptive time-scale separation (null when off): offsets at the last
    // force evaluation, and the device words {largest displacement since it
    // (FP64 bits), steps since it, evaluate on this step, first step pending}
    R *off_eval;
    unsigned long long *adapt;  // ADAPT_WORDS words; the fifth counts the evaluations
    // internal viscosity (null when off): per-node indicator of the cell
    // interiors and the toggle counts it is built from; relaxation rate inside
    uint8_t *ind;
    int *tog;
    R omega_in;
    // Lees-Edwards boundary along z (le = 0: off): image velocity, the
    // device step counter of the displacement D_n = U n mod nx, the second
    // population array of the two-array streaming and the post-collision
    // moments (rho, u) of the planes z = 0 and z = nz - 1 ([2][ny][nx][4])
    int le;
    double le_U;
    long long *le_n;
    void *f2;
    R *le_aux;
    R *csp;                    // ncell*6 centroid of the last re-base as R hi (3), lo (3)
    int spread_all_nodes;      // 0: F = g + sum at fluid nodes, 0 at walls; 1: the sum at every node
    unsigned *status;
    // staged collision: tiles {first row, rows, y, z of the first row} of
    // wall-free rows (x-lines, row index y + ny z; a tile's rows lie in one
    // z-plane) and the other rows that hold fluid
    const int4 *rtiles;
    int ntiles, tile_rows, tile_stages, tile_grid, tile_smem;
    const int *erows;
    int nerows;
    // 16-bit storage: per row (x-line, index y + ny z) the reference values
    // (P, M) of the stored populations (see k_lattice.cu); all zero when no
    // reference is set.  Null for 4- and 8-byte storage.
    const float2 *rref;
    int node_pairs;            // 16-bit storage, nx even: PAIR_* bits, kernels that take two nodes per thread
    int stalled_wait_test;     // staged collision: first wait on a barrier nothing completes (HEMO_OPT_TEST_STALLED_WAIT)
    int wide_index;            // lattice kernels: 64-bit population indices on any lattice (HEMO_OPT_WIDE_INDEX)
    // interpolation staging by tensor copies: the host-side tensor map of u
    // (CUtensorMap, 4-D: x, y, z, component) and the array it describes;
    // null when off (FP64, or nx not a multiple of 4)
    const void *u_tmap;
    const void *u_tmap_base;
    // a buffer whose contents are dead: the kernel drops its full 128-byte
    // lines from L2 without writing them back (null / 0 = nothing to drop)
    void *dead;
    long long dead_lines;
    // recording for the reverse sweep (null in plain steps)
    R *rec;                    // [4][N] collision density and velocity at fluid nodes; when set the
                               // moments kernel also writes the wall velocity into u at wall nodes
    R *off_rec;                // nv*3 re-based offsets as the membrane forces saw them
};

// Adjoint (reverse-mode) state of one step; all lattice arrays natural
// layout, SoA, in R.  Gradient slots: per mesh type t: 4t + (k_link, k_bend,
// k_area, k_volume); then wall-velocity scale, g_x, g_y, g_z.
template <typename R> struct AdjView {
    const R *rec;     // [4][N] collision density and velocity of step n (fluid nodes)
    const R *rho1;    // N: density of f_{n+1} (fluid nodes)
    const R *up;      // [3][N] u_{n+1} as the forward step wrote it (wall velocity at walls)
    R *amom;          // [4][N] moments transpose per node: lamu / rho' (3), -(lamu . u') / rho'
    R *lamf_in;       // 19*N adjoint of f_{n+1}, without the moments term
    R *lamf_out;      // 19*N adjoint of f_n
    R *lamu;          // [3][N] adjoint of u_{n+1}
    R *lamF;          // [3][N] adjoint of F_n
    R *lamX;          // nv*3 adjoint of the vertex positions
    R *lamFv;         // nv*3 adjoint of the membrane forces
    double *grad;     // gradient accumulators (device)
    int ntypes;
};

// launchers (R = double for HEMO_F64, float otherwise)
template <typename R> void launch_collide(const View<R> &v, int precision, int parity, cudaStream_t st);
template <typename R> void launch_hold_bins(const View<R> &v, cudaStream_t st);
// adaptive separation: decide whether this step evaluates the membrane forces
void launch_adapt_decide(unsigned long long *adapt, double tol, int every, cudaStream_t st);
// inside/outside indicator at the current vertex positions into v.ind
template <typename R> void launch_inside(const View<R> &v, cudaStream_t st);
// Lees-Edwards boundary: two-array collision and streaming, the coupling of
// the vertices in the extra bin, and the step counter of the displacement
template <typename R> void launch_le_lattice(const View<R> &v, int precision, cudaStream_t st);
template <typename R> void launch_le_spread(const View<R> &v, cudaStream_t st);
template <typename R> void launch_le_interp(const View<R> &v, cudaStream_t st);
void launch_le_advance(long long *n, cudaStream_t st);
// allows the staged collision kernels of a precision `bytes` of dynamic shared memory
cudaError_t set_tile_smem_limit(int precision, int bytes);
template <typename R> void launch_moments(const View<R> &v, int precision, int parity, cudaStream_t st);
// 16-bit storage: the rows' reference (P, M) from a velocity field ([n][3]
// double, device) and the re-storing of natural-order populations from one
// reference table to another (null = zero reference)
void launch_row_reference(const View<float> &v, const double *u0, float2 *rref, cudaStream_t st);
void launch_reencode(const View<float> &v, int precision, const float2 *from, const float2 *to, cudaStream_t st);
template <typename R> void launch_init_equilibrium(const View<R> &v, int precision, const double *u_dev, cudaStream_t st);
template <typename R> void launch_populations_out(const View<R> &v, int precision, int parity, double *out, cudaStream_t st);
template <typename R> void launch_rho_out(const View<R> &v, int precision, int parity, R *out, cudaStream_t st);
template <typename R> void launch_u_out(const View<R> &v, R *out, cudaStream_t st);
void launch_build_links(int nx, int ny, int nz, const int *per, uint8_t *ntype, uint64_t *links, cudaStream_t st);

// mode 0 (the step): re-base the offsets, membrane forces into Fv, and the
// vertices' anchors, bin keys and bin counts (counts zeroed beforehand);
// mode 1: per-cell statistics into stats (6 per cell), no writes to the state
template <typename R> void launch_cell_forces(const View<R> &v, int mode, double *stats, cudaStream_t st);
template <typename R> cudaError_t set_cell_smem_limit(size_t bytes);
template <typename R> size_t cell_smem_bytes(int max_nv, int max_nt, int max_ne) {
    return (4 * (size_t)max_nv + 5 * (size_t)max_nt + 4 * (size_t)max_ne) * sizeof(R);
}
template <typename R> void launch_bins(const View<R> &v, cudaStream_t st, bool stable);
// the bin ranges and the (unstable) order once the step's membrane kernel
// has written the anchors, keys and counts
template <typename R> void launch_bin_ranges(const View<R> &v, cudaStream_t st);
template <typename R> void launch_spread(const View<R> &v, cudaStream_t st);
template <typename R> void launch_interpolate(const View<R> &v, cudaStream_t st);
template <typename R> void launch_verts_out(const View<R> &v, double *X, double *F, cudaStream_t st);
template <typename R> void launch_set_vertices(const View<R> &v, const double *X, cudaStream_t st);

// adjoint step (natural-layout arrays) and checkpoints
template <typename R> void launch_copy_natural(const View<R> &v, int precision, int layout, R *out, cudaStream_t st);
template <typename R> void launch_restore_natural(const View<R> &v, int precision, int layout, const R *in, cudaStream_t st);
template <typename R> void launch_adj_moments(const View<R> &v, const AdjView<R> &a, cudaStream_t st);
template <typename R> void launch_adj_collide(const View<R> &v, const AdjView<R> &a, cudaStream_t st);
template <typename R> void launch_cell_adjoint(const View<R> &v, const AdjView<R> &a, cudaStream_t st);
template <typename R> cudaError_t set_cell_adjoint_smem_limit(size_t bytes);
template <typename R> size_t cell_adjoint_smem_bytes(int max_nv, int max_nt) { return (9 * (size_t)max_nv + 8 * (size_t)max_nt) * sizeof(R); }
// FP32 gather form of the membrane adjoint: positions, direction, triangle
// and edge records with their derivatives, 16 bytes each; used while it fits
// the largest shared-memory allocation of a CTA
inline size_t cell_adjoint_gather_bytes(int max_nv, int max_nt, int max_ne) {
    return 8 * ((size_t)max_nv + (size_t)max_nt + (size_t)max_ne) * sizeof(float);
}
constexpr size_t CELL_ADJ_GATHER_MAX_SMEM = 227 * 1024;
cudaError_t set_cell_adjoint_gather_smem_limit(size_t bytes);
template <typename R>
void launch_vertex_field(const View<R> &v, const R *field, const R *vec, R *out_grad, R *out_interp, cudaStream_t st);
template <typename R>
void launch_deformation_loss(const View<R> &v, const double *c0, double *cell_loss, R *dLdX, cudaStream_t st);

// Sums at FP64-level precision.  In the FP64 path a plain double; in FP32 a
// two-word accumulator (hi + lo, each addition by Knuth's TwoSum),
// so the loops over triangles and vertices do no FP64 arithmetic (slow on
// this GPU) and only the per-warp totals are combined in FP64.
template <typename R> struct Acc {
    double s = 0;
    __device__ void add(double x) { s += x; }
    __device__ void add_shfl(int o) { s += __shfl_down_sync(0xffffffffu, s, o); }
    __device__ double value() const { return s; }
};
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ void add(float x) {
        const float sum = hi + x, bp = sum - hi;
        lo += (hi - (sum - bp)) + (x - bp);
        hi = sum;
    }
    __device__ void add_shfl(int o) {
        const float h = __shfl_down_sync(0xffffffffu, hi, o), l = __shfl_down_sync(0xffffffffu, lo, o);
        add(h);
        lo += l;
    }
    __device__ double value() const { return (double)hi + (double)lo; }
};

// Drops this thread's share of the dead buffer's L2 lines (discard.global.L2:
// the lines are invalidated without write-back, so data that no kernel will
// read again costs no DRAM writes when it would be evicted).
template <typename R>
__device__ __forceinline__ void drop_dead_lines(const View<R> &v) {
    if (!v.dead_lines) return;
    const long long bs = (long long)blockDim.x * blockDim.y * blockDim.z;
    const long long stride = (long long)gridDim.x * gridDim.y * gridDim.z * bs;
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    const long long t = threadIdx.x + (long long)blockDim.x * (threadIdx.y + (long long)blockDim.y * threadIdx.z);
    for (long long l = b * bs + t; l < v.dead_lines; l += stride)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"((char *)v.dead + 128 * l) : "memory");
}

// sets the message returned by hemo_last_error() on the calling thread
void set_last_error(const char *msg);

// index offsets of a node's +/- neighbours per axis (periodic wrap built in;
// offsets across a non-periodic edge are never used: those links are walls)
struct Nbr {
    int xp, xm, yp, ym, zp, zm;  // index offsets to the +/- neighbour per axis (wrapped)
    __device__ __forceinline__ int of(int ccx, int ccy, int ccz) const {
        return (ccx > 0 ? xp : (ccx < 0 ? xm : 0)) + (ccy > 0 ? yp : (ccy < 0 ? ym : 0)) +
               (ccz > 0 ? zp : (ccz < 0 ? zm : 0));
    }
};

template <typename R>
__device__ __forceinline__ Nbr nbr_at(const View<R> &v, int x, int y, int z) {
    const int sxy = v.nx * v.ny;
    Nbr o;
    o.xp = (x == v.nx - 1) ? -(v.nx - 1) : 1;
    o.xm = (x == 0) ? (v.nx - 1) : -1;
    o.yp = (y == v.ny - 1) ? -(v.ny - 1) * v.nx : v.nx;
    o.ym = (y == 0) ? (v.ny - 1) * v.nx : -v.nx;
    o.zp = (z == v.nz - 1) ? -(v.nz - 1) * sxy : sxy;
    o.zm = (z == 0) ? (v.nz - 1) * sxy : -sxy;
    return o;
}

template <typename R>
__device__ __forceinline__ Nbr make_nbr(const View<R> &v, int n) {
    const int r = n / v.nx;
    return nbr_at(v, n % v.nx, r % v.ny, r / v.ny);
}

// mbarrier and async-proxy helpers (completion of bulk and tensor copies
// into shared memory; every wait is bounded)
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

// waits for the phase with the given parity; gives up after limit_ns
// (about a second by default)
__device__ inline bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 256; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Lattice kernels over all nodes use a grid of (x chunks of NODE_BX) x (y
// groups of NODE_BY) x z with blocks of NODE_BX x NODE_BY threads: node
// coordinates come without integer division and a warp covers 32
// consecutive nodes of one x-row.  The velocity pass (few registers, many
// CTAs per SM) takes y groups of MOM_BY: smaller CTAs, measured faster.
constexpr int NODE_BX = 32, NODE_BY = 8, MOM_BY = 4;

__device__ __forceinline__ int link_code(uint64_t lk, int i) { return (int)((lk >> (2 * i)) & 3u); }

// periodic wrap of a lattice coordinate
__host__ __device__ __forceinline__ int wrap(int j, int n) {
    int r = j % n;
    return r < 0 ? r + n : r;
}

// Anchor of a coordinate X = c + o (c the FP64 centroid, o the offset):
// j = floor(X), t = X - j.  FP32 path: c arrives split into two floats
// (c = ch + cl to 48 bits) and X is formed as a two-float sum, which keeps
// t to FP32 precision without FP64 arithmetic.
__device__ __forceinline__ void anchor_of(float ch, float cl, float o, int &j, float &t) {
    const float sum = ch + o, bp = sum - ch;
    const float err = ((ch - (sum - bp)) + (o - bp)) + cl;
    const float fl = floorf(sum);
    j = (int)fl;
    t = (sum - fl) + err;  // sum - fl is exact
    if (t >= 1.f) {
        t -= 1.f;
        ++j;
    } else if (t < 0.f) {
        t += 1.f;
        --j;
    }
}
__device__ __forceinline__ void anchor_of(double c, double, double o, int &j, double &t) {
    const double X = c + o, fl = floor(X);
    j = (int)fl;
    t = X - fl;
}

// z = c + o as R (Lees-Edwards binning: the plane crossing is decided on it)
__device__ __forceinline__ float anchor_z_unwrapped(float ch, float cl, float o) {
    int j;
    float t;
    anchor_of(ch, cl, o, j, t);
    return (float)j + t;
}
__device__ __forceinline__ double anchor_z_unwrapped(double c, double, double o) { return c + o; }

// displacement of the Lees-Edwards image above at the current step, in [0, nx)
template <typename R>
__device__ __forceinline__ double le_shift(const View<R> &v) {
    double D = fmod(v.le_U * (double)(*v.le_n), (double)v.nx);
    return D < 0 ? D + v.nx : D;
}

// Stencil anchor (wrapped floor and fraction per axis), bin key and bin
// count of vertex g at X = (ch + cl) + o; flags a vertex outside a
// non-periodic axis.  Bin counts are added once per group of lanes with the
// same key.
template <typename R>
__device__ __forceinline__ void bin_vertex(const View<R> &v, size_t g, const R *ch, const R *cl, const R *o) {
    const int dims[3] = {v.nx, v.ny, v.nz};
    int b[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int j;
        R t;
        anchor_of(ch[d], cl[d], o[d], j, t);
        if (v.per[d]) {
            j = wrap(j, dims[d]);
        } else if (j < 0 || j >= dims[d]) {
            atomicOr(v.status, ST_DOMAIN);
        }
        v.anc_i[3 * g + d] = j;
        v.anc_t[3 * g + d] = t;
        const int jc = j < 0 ? 0 : (j >= dims[d] ? dims[d] - 1 : j);
        b[d] = jc / BLK;
    }
    int key = b[0] + v.nb[0] * (b[1] + v.nb[1] * b[2]);
    if (v.le) {  // Lees-Edwards: stencils reaching across z = 0 or z = nz go to the extra bin, with z unwrapped
        const R zu = anchor_z_unwrapped(ch[2], cl[2], o[2]);
        const int jz = (int)floor(zu);
        if (jz < 1 || jz + 2 >= v.nz) {
            key = v.nbins;
            v.anc_i[3 * g + 2] = jz;
            v.anc_t[3 * g + 2] = zu - R(jz);
        }
    }
    v.key[g] = key;
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, key);
    if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(v.counts + key, __popc(grp));
}

}  // namespace hemo
