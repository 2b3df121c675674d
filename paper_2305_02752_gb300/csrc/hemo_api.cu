// Host side of the C ABI declared in include/hemo.h: simulation state,
// device allocation, mesh preprocessing (edge tables, rest geometry), the
// per-step kernel sequence captured once per parity as a CUDA graph, status
// handling and read-out.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <string>
#include <map>
#include <unordered_map>
#include <vector>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include "hemo_internal.cuh"

using namespace hemo;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

// NVTX ranges (no-ops unless a profiler is attached): one per API call that
// launches work, and one per phase of the step where its kernels are
// enqueued (inside a graph capture: once per captured variant; the device
// time per phase comes from the event nodes of hemo_set_phase_timing)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
const char *const PHASE_NAMES[HEMO_NUM_PHASES] = {"membrane", "bins", "spread", "collide", "moments", "interp"};

#define HEMO_CU(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(HEMO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct HostMesh {
    int nv = 0, nt = 0, ne = 0;
    std::vector<int> tri, edge;
    std::vector<double> L0, th0, At0;
    double A0 = 0, V0 = 0;
    double k_link = 0, k_bend = 0, k_area = 0, k_volume = 0, kbt = 0, persistence = 1, max_strain = 1;
    double k_local = 0, theta_m = 0;
};

// Edge table of a closed oriented triangle mesh: edges numbered by first
// appearance (triangles in order, directed edges t0t1, t1t2, t2t0); the first
// triangle gives (v0, v1, a), the second (necessarily traversing v1 -> v0)
// gives b.  Returns false if the mesh is not a consistently oriented closed
// 2-manifold.
bool build_edge_table(int nv, const std::vector<int> &tri, std::vector<int> &edge) {
    const int nt = (int)tri.size() / 3;
    std::unordered_map<long long, int> id;
    id.reserve(3 * nt);
    edge.clear();
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            const int a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3], o = tri[3 * t + (k + 2) % 3];
            const long long key = (long long)std::min(a, b) * nv + std::max(a, b);
            auto it = id.find(key);
            if (it == id.end()) {
                id.emplace(key, (int)(edge.size() / 4));
                edge.insert(edge.end(), {a, b, o, -1});
            } else {
                int *e = &edge[4 * it->second];
                if (e[0] != b || e[1] != a || e[3] != -1) return false;
                e[3] = o;
            }
        }
    for (size_t e = 0; e < edge.size() / 4; ++e)
        if (edge[4 * e + 3] < 0) return false;
    return true;
}

struct D3 {
    double x, y, z;
};
D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
D3 crs(D3 a, D3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double dt3(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// smallest stride >= n/32 + 1 that is coprime with n (1 for small n)
int coprime_stride(int n) {
    auto gcd = [](int a, int b) {
        while (b) {
            int t = a % b;
            a = b;
            b = t;
        }
        return a;
    };
    for (int st = n / 32 + 1; st < n; ++st)
        if (gcd(st, n) == 1) return st;
    return 1;
}


}  // namespace

void hemo::set_last_error(const char *msg) { g_err = msg; }

// device buffers of the reverse sweep (grown on demand, kept for reuse)
constexpr size_t TILE_NODES3 = (size_t)(BLK + 3) * (BLK + 3) * (BLK + 3);  // nodes of a bin's spreading tile

struct AdjBuffers {
    void *lamf_in = nullptr, *lamf_out = nullptr, *lamu = nullptr, *lamF = nullptr, *amom = nullptr;
    void *lamX = nullptr, *lamFv = nullptr, *grad = nullptr;
    void *fin_f = nullptr, *fin_u = nullptr, *fin_ctr = nullptr, *fin_off = nullptr, *cell_loss = nullptr, *dldx = nullptr;
    // per step of a segment
    void *seg_rec = nullptr, *seg_F = nullptr, *seg_u = nullptr, *seg_off = nullptr, *seg_Fv = nullptr;
    void *seg_anc_i = nullptr, *seg_anc_t = nullptr, *seg_perm = nullptr, *seg_start = nullptr;
    size_t sz_lamf_in = 0, sz_lamf_out = 0, sz_lamu = 0, sz_lamF = 0, sz_amom = 0, sz_lamX = 0, sz_lamFv = 0, sz_grad = 0;
    size_t sz_fin_f = 0, sz_fin_u = 0, sz_fin_ctr = 0, sz_fin_off = 0, sz_cell_loss = 0, sz_dldx = 0;
    size_t sz_seg_rec = 0, sz_seg_F = 0, sz_seg_u = 0, sz_seg_off = 0, sz_seg_Fv = 0;
    size_t sz_seg_anc_i = 0, sz_seg_anc_t = 0, sz_seg_perm = 0, sz_seg_start = 0;
};

struct hemo_sim {
    int precision = 0;
    // tensor map of u for the interpolation's staging (FP32 arithmetic, nx
    // a multiple of 4, unless HEMO_OPT_NODE_STAGING)
    CUtensorMap u_tmap;
    bool u_tma = false;
    int nx = 0, ny = 0, nz = 0;
    long long N = 0;
    int per[3] = {1, 1, 1};
    double tau = 1, g[3] = {0, 0, 0}, uw[2][3] = {{0, 0, 0}, {0, 0, 0}};
    cudaStream_t stream = nullptr;
    hemo_alloc_fn alloc = nullptr;
    hemo_free_fn release = nullptr;
    void *ctx = nullptr;
    std::vector<void *> allocs;
    // lattice
    void *f = nullptr;
    uint8_t *ntype = nullptr;
    uint64_t *links = nullptr;
    void *F = nullptr, *u = nullptr;
    unsigned options = 0;
    float2 *rref = nullptr;       // 16-bit storage: the rows' reference (P, M), see k_lattice.cu
    // staged collision (tiles of wall-free rows), see plan_rows
    int4 *rtiles = nullptr;
    int *erows = nullptr;
    int ntiles = 0, nerows = 0, tile_rows = 0, tile_stages = 0, tile_grid = 0, tile_smem = 0;
    // cells (host until finalised)
    std::vector<HostMesh> meshes;
    std::vector<int> cell_type, cell_first, vcell;
    std::vector<double> X0;
    int nv = 0, ncell = 0, max_nv = 0, max_nt = 0, max_ne = 0, nsm = 1;
    bool finalized = false;
    long long steps_done = 0;
    // device cells and bins
    double *ctr = nullptr;
    void *off = nullptr, *Fv = nullptr;
    int *vcell_d = nullptr, *cell_first_d = nullptr, *cell_type_d = nullptr;
    void *meshes_d = nullptr;
    int nb[3] = {1, 1, 1}, nbins = 1;
    int *key = nullptr, *counts = nullptr, *start = nullptr, *cursor = nullptr, *perm_raw = nullptr, *perm = nullptr;
    int *anc_i = nullptr;
    void *anc_t = nullptr;
    void *tiles = nullptr;
    // status
    unsigned *status = nullptr;
    unsigned *status_host = nullptr;
    cudaEvent_t ev = nullptr;
    bool ev_pending = false;
    unsigned sticky = 0;
    // time-scale separation and vertex integrator (Sec. 2.6)
    int force_every = 1;          // membrane forces on every force_every-th step, held in between
    int integrator = HEMO_EULER;
    long long ts_origin = 0;      // step count at which the setting was made
    long long evals_host = 0;     // membrane-force evaluations of constant-schedule steps (adaptive ones: adapt[4])
    bool have_prev = false;       // Uprev holds the previous step's vertex velocity
    void *Uprev = nullptr;
    void *csp = nullptr;          // per cell: centroid of the last re-base as R hi, lo
    // adaptive separation: tolerance (< 0: off), offsets at the last force
    // evaluation and the device decision words (see View)
    double force_tol = -1.0;
    void *off_eval = nullptr;
    unsigned long long *adapt = nullptr;
    // internal viscosity (Sec. 1, Sec. 3): ratio of the viscosity inside cells
    double visc_ratio = 1.0;      // 1: off
    uint8_t *ind = nullptr;       // N: inside a cell
    int *tog = nullptr;           // N: toggle counts (zero between steps)
    // Lees-Edwards boundary along z (Sec. 2.5)
    bool has_walls = false;
    bool le = false;
    double le_U = 0;
    void *f2 = nullptr, *le_aux = nullptr;
    long long *le_n = nullptr;
    // graphs, one per step variant: parity + 2 force step + 4 integrator mode
    // (0..11), and with the adaptive separation 12 + parity + 2 integrator mode
    cudaStream_t cap = nullptr;
    static constexpr int NGRAPH = 18;
    cudaGraphExec_t graph[NGRAPH] = {};
    int graph_kernels[NGRAPH] = {};
    int last_graph = -1;
    // staging for read-out
    void *staging = nullptr;
    size_t staging_bytes = 0;
    // phase timing
    bool timing = false;
    cudaEvent_t tev[HEMO_NUM_PHASES + 1] = {};
    // differentiation form
    bool rec = false;
    int ck_every = 0;
    long long rec_start = 0;
    std::vector<void *> ck_f, ck_ctr, ck_off;
    double *c0 = nullptr;
    AdjBuffers adj;
    std::map<long long, cudaGraphExec_t> seg_graphs;  // reverse-sweep segments by (length, buffer parity)
};

namespace {

void *dalloc(hemo_sim *s, size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    void *p = nullptr;
    if (s->alloc) {
        p = s->alloc(bytes, s->ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) s->allocs.push_back(p);
    return p;
}

void dfree(hemo_sim *s, void *p) {
    if (!p) return;
    auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
    if (it != s->allocs.end()) s->allocs.erase(it);
    if (s->release) s->release(p, s->ctx);
    else if (!s->alloc) cudaFree(p);
}

bool is_f64(const hemo_sim *s) { return s->precision == HEMO_F64; }
size_t rsize(const hemo_sim *s) { return is_f64(s) ? 8 : 4; }
size_t tsize(const hemo_sim *s) {
    switch (s->precision) {
        case HEMO_F64: return 8;
        case HEMO_F32: return 4;
        default: return 2;
    }
}

int status_code(unsigned st) {
    if (st & ST_NUMERIC) return fail(HEMO_ERR_NUMERIC, "device status: non-finite or |u| > 0.3 velocity, or a link stretched past its maximum strain");
    if (st & ST_DOMAIN) return fail(HEMO_ERR_DOMAIN, "device status: a vertex left the lattice across a non-periodic axis");
    if (st & ST_TIMEOUT) return fail(HEMO_ERR_CUDA, "device status: a copy pipeline wait timed out");
    if (st & ST_BOUNDS) return fail(HEMO_ERR_CUDA, "device status: an index failed its bounds check (bounds-checked build)");
    return HEMO_OK;
}

int ensure_staging(hemo_sim *s, size_t bytes) {
    if (s->staging_bytes >= bytes) return HEMO_OK;
    HEMO_CU(cudaStreamSynchronize(s->stream));
    dfree(s, s->staging);
    s->staging = dalloc(s, bytes);
    s->staging_bytes = s->staging ? bytes : 0;
    if (!s->staging) return fail(HEMO_ERR_OOM, "staging buffer allocation failed");
    return HEMO_OK;
}

// The tensor map of u ([3][nz][ny][nx] FP32, described as a 4-D tensor x,
// y, z, component) for the interpolation's staging, box 16 x 11 x 11 x 3
// (see k_ibm.cu).  False (node-by-node staging) for FP64, for nx not a
// multiple of 4 (row strides must be multiples of 16 bytes), on request,
// or when the driver does not provide the encoder.
bool encode_u_tmap(hemo_sim *s) {
    if (s->precision == HEMO_F64 || (s->options & HEMO_OPT_NODE_STAGING) || s->nx % 4 != 0 || !s->u) return false;
    if (((uintptr_t)s->u & 15) != 0) return false;
    using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)s->nx, (cuuint64_t)s->ny, (cuuint64_t)s->nz, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)s->nx * 4, (cuuint64_t)s->nx * s->ny * 4, (cuuint64_t)s->N * 4};
    const cuuint32_t box[4] = {16, 11, 11, 3}, estr[4] = {1, 1, 1, 1};
    const CUresult r = reinterpret_cast<EncodeFn>(fn)(&s->u_tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, s->u, dims, strides,
                                                      box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <typename R>
View<R> make_view(hemo_sim *s) {
    View<R> v{};
    v.nx = s->nx;
    v.ny = s->ny;
    v.nz = s->nz;
    v.N = s->N;
    for (int d = 0; d < 3; ++d) v.per[d] = s->per[d];
    v.f = s->f;
    v.ntype = s->ntype;
    v.links = s->links;
    v.F = (R *)s->F;
    v.u = (R *)s->u;
    v.omega = R(1.0 / s->tau);
    v.rtiles = s->rtiles;
    v.ntiles = s->ntiles;
    v.tile_rows = s->tile_rows;
    v.tile_stages = s->tile_stages;
    v.tile_grid = s->tile_grid;
    v.tile_smem = s->tile_smem;
    v.erows = s->erows;
    v.nerows = s->nerows;
    v.rref = s->rref;
    // 16-bit storage, nx even: the velocity pass two nodes per thread (the
    // faster form, measured); the collision two nodes per thread only on
    // request (the per-node kernel is faster on odd steps and as fast on even)
    v.node_pairs = 0;
    if (tsize(s) == 2 && (s->nx % 2) == 0 && !(s->options & HEMO_OPT_NODE_COLLISION))
        v.node_pairs = PAIR_MOMENTS | ((s->options & HEMO_OPT_PAIR_COLLISION) ? PAIR_COLLIDE : 0);
    v.stalled_wait_test = (s->options & HEMO_OPT_TEST_STALLED_WAIT) ? 1 : 0;
    v.wide_index = (s->options & HEMO_OPT_WIDE_INDEX) ? 1 : 0;
    v.u_tmap = s->u_tma ? (const void *)&s->u_tmap : nullptr;
    v.u_tmap_base = s->u_tma ? s->u : nullptr;
    for (int d = 0; d < 3; ++d) {
        v.g[d] = R(s->g[d]);
        v.uw[0][d] = R(0);
        v.uw[1][d] = R(0);
        v.uw[2][d] = R(s->uw[0][d]);
        v.uw[3][d] = R(s->uw[1][d]);
    }
    v.nv = s->nv;
    v.ncell = s->ncell;
    v.ctr = s->ctr;
    v.off = (R *)s->off;
    v.Fv = (R *)s->Fv;
    v.vcell = s->vcell_d;
    v.cell_first = s->cell_first_d;
    v.cell_type = s->cell_type_d;
    v.meshes = (const MeshDev<R> *)s->meshes_d;
    v.max_nv = s->max_nv;
    v.max_nt = s->max_nt;
    v.max_ne = s->max_ne;
    v.nsm = s->nsm;
    for (int d = 0; d < 3; ++d) v.nb[d] = s->nb[d];
    v.nbins = s->nbins;
    v.key = s->key;
    v.counts = s->counts;
    v.start = s->start;
    v.cursor = s->cursor;
    v.perm_raw = s->perm_raw;
    v.perm = s->perm;
    v.anc_i = s->anc_i;
    v.anc_t = (R *)s->anc_t;
    v.tiles = (R *)s->tiles;
    v.status = s->status;
    v.integ = 0;
    v.Uprev = (R *)s->Uprev;
    v.csp = (R *)s->csp;
    if (s->force_tol >= 0) {
        v.off_eval = (R *)s->off_eval;
        v.adapt = s->adapt;
    }
    if (s->visc_ratio != 1.0) {
        v.ind = s->ind;
        v.tog = s->tog;
        v.omega_in = R(1.0 / (0.5 + s->visc_ratio * (s->tau - 0.5)));
    }
    if (s->le) {
        v.le = 1;
        v.le_U = s->le_U;
        v.le_n = s->le_n;
        v.f2 = s->f2;
        v.le_aux = (R *)s->le_aux;
    }
    return v;
}

// One coupled step.  force: 1 evaluate the membrane forces, 0 hold the last
// ones (Sec. 2.6), 2 decide on the device (adaptive separation); v.integ
// selects the vertex integrator.
template <typename R>
void enqueue_step(hemo_sim *s, const View<R> &v, int parity, int force, cudaStream_t st) {
    auto mark = [&](int k) {
        if (s->timing) cudaEventRecordWithFlags(s->tev[k], st, cudaEventRecordExternal);
        if (k != HEMO_PHASE_MEMBRANE) nvtxRangePop();
        if (k != HEMO_NUM_PHASES) nvtxRangePushA(PHASE_NAMES[k]);
    };
    mark(HEMO_PHASE_MEMBRANE);
    if (s->ncell) {
        // (the bin counts start at zero: the previous scan reset them)
        if (force == 2) {  // adaptive: both kernels, each runs only on its kind of step
            launch_adapt_decide(v.adapt, s->force_tol, s->force_every, st);
            launch_cell_forces<R>(v, 0, nullptr, st);
            launch_hold_bins<R>(v, st);
        } else if (force) {
            launch_cell_forces<R>(v, 0, nullptr, st);  // re-base, A and V, F_v at X^n; anchors and bin counts
        } else {
            launch_hold_bins<R>(v, st);  // F_v held: anchors and bin counts only
        }
    }
    if (v.ind) launch_inside<R>(v, st);  // cell interiors at X^n (internal viscosity)
    mark(HEMO_PHASE_BINS);
    if (s->ncell) launch_bin_ranges<R>(v, st);  // counting sort by block
    mark(HEMO_PHASE_SPREAD);
    if (s->ncell) launch_spread<R>(v, st);  // F = g + sum F_v delta
    if (s->ncell && v.le) launch_le_spread<R>(v, st);  // vertices at the Lees-Edwards plane
    mark(HEMO_PHASE_COLLIDE);
    if (v.le) {  // Lees-Edwards: two-array collision and streaming, then the coupling at the plane
        launch_le_lattice<R>(v, s->precision, st);
        mark(HEMO_PHASE_MOMENTS);
        mark(HEMO_PHASE_INTERP);
        if (s->ncell) {
            launch_interpolate<R>(v, st);
            launch_le_interp<R>(v, st);
        }
        launch_le_advance(v.le_n, st);
        mark(HEMO_NUM_PHASES);
        return;
    }
    View<R> vc = v;  // the spreading tiles are dead once F is gathered
    if (s->ncell) {
        vc.dead = s->tiles;
        vc.dead_lines = (long long)(rsize(s) * 3 * (size_t)TILE_NODES3 * s->nbins / 128);
    }
    launch_collide<R>(vc, s->precision, parity, st);  // BGK + Guo force + AA streaming
    mark(HEMO_PHASE_MOMENTS);
    launch_moments<R>(v, s->precision, parity, st);  // post-streaming u (with F/2)
    mark(HEMO_PHASE_INTERP);
    View<R> vi = v;  // F is dead once the moments have read it
    if (!v.rec) {
        vi.dead = v.F;
        vi.dead_lines = (long long)(rsize(s) * 3 * (size_t)s->N / 128);
    }
    if (s->ncell) launch_interpolate<R>(vi, st);  // X^{n+1} = X^n + I[u](X^n) (Euler or Adams-Bashforth)
    mark(HEMO_NUM_PHASES);
}

template <typename R>
int finalize_impl(hemo_sim *s) {
    const size_t rs = sizeof(R);
    const int nv = s->nv, nc = s->ncell;
    s->ctr = (double *)dalloc(s, sizeof(double) * 3 * std::max(nc, 1));
    s->off = dalloc(s, rs * 3 * std::max(nv, 1));
    s->Fv = dalloc(s, rs * 3 * std::max(nv, 1));
    s->vcell_d = (int *)dalloc(s, sizeof(int) * std::max(nv, 1));
    s->cell_first_d = (int *)dalloc(s, sizeof(int) * std::max(nc, 1));
    s->cell_type_d = (int *)dalloc(s, sizeof(int) * std::max(nc, 1));
    s->meshes_d = dalloc(s, sizeof(MeshDev<R>) * MAX_TYPES);
    s->key = (int *)dalloc(s, sizeof(int) * std::max(nv, 1));
    s->perm_raw = (int *)dalloc(s, sizeof(int) * std::max(nv, 1));
    s->perm = (int *)dalloc(s, sizeof(int) * std::max(nv, 1));
    s->anc_i = (int *)dalloc(s, sizeof(int) * 3 * std::max(nv, 1));
    s->anc_t = dalloc(s, rs * 3 * std::max(nv, 1));
    // one more bin than the lattice has: the vertices at the Lees-Edwards plane
    s->counts = (int *)dalloc(s, sizeof(int) * (s->nbins + 1));
    s->cursor = (int *)dalloc(s, sizeof(int) * (s->nbins + 1));
    s->start = (int *)dalloc(s, sizeof(int) * (s->nbins + 2));
    s->tiles = dalloc(s, rs * 3 * TILE_NODES3 * s->nbins);
    s->Uprev = dalloc(s, rs * 3 * std::max(nv, 1));
    s->csp = dalloc(s, rs * 6 * std::max(nc, 1));
    if (!s->tiles || !s->Uprev || !s->csp || !s->ctr || !s->off || !s->Fv || !s->vcell_d || !s->cell_first_d || !s->cell_type_d || !s->meshes_d ||
        !s->key || !s->perm_raw || !s->perm || !s->anc_i || !s->anc_t ||
        !s->counts || !s->cursor || !s->start)
        return fail(HEMO_ERR_OOM, "device allocation of cell and bin buffers failed");
    cudaStream_t st = s->stream;
    HEMO_CU(cudaMemsetAsync(s->start, 0, sizeof(int) * (s->nbins + 2), st));
    HEMO_CU(cudaMemsetAsync(s->counts, 0, sizeof(int) * (s->nbins + 1), st));
    HEMO_CU(cudaMemsetAsync(s->Fv, 0, rs * 3 * std::max(nv, 1), st));

    // mesh tables
    std::vector<MeshDev<R>> md(MAX_TYPES);
    for (size_t t = 0; t < s->meshes.size(); ++t) {
        const HostMesh &m = s->meshes[t];
        int *dtri = (int *)dalloc(s, sizeof(int) * m.tri.size());
        int *dedge = (int *)dalloc(s, sizeof(int) * m.edge.size());
        int *detri = (int *)dalloc(s, sizeof(int) * 2 * (size_t)m.ne);
        R *dL0 = (R *)dalloc(s, rs * m.ne);
        R *dth0 = (R *)dalloc(s, rs * m.ne);
        int4 *dtri4 = (int4 *)dalloc(s, sizeof(int4) * (size_t)m.nt);
        if (!dtri || !dedge || !detri || !dL0 || !dth0 || !dtri4)
            return fail(HEMO_ERR_OOM, "device allocation of mesh tables failed");
        // processing order: triangles and edges sorted by their smallest
        // vertex id, so that the lanes of a warp (consecutive vertices in the
        // gather, consecutive items in the triangle and edge passes) load
        // nearby shared-memory records (measured: membrane kernel 1163 ->
        // 976 us on the pipe against the earlier order that spread a warp
        // over far-apart mesh parts, made for scattering atomics).  The FP64
        // adjoint, which still scatters with atomics, walks the same tables
        // with a coprime stride (MeshDev::tstride, estride).
        std::vector<int> edge_p(4 * (size_t)m.ne), tri_p(3 * (size_t)m.nt), tpos(m.nt), etri_p(2 * (size_t)m.ne);
        std::vector<R> invL0(m.ne), th0(m.ne);
        std::vector<R> At0_p(m.nt);
        std::vector<int> tord(m.nt), eord(m.ne);
        for (int q = 0; q < m.nt; ++q) tord[q] = q;
        for (int q = 0; q < m.ne; ++q) eord[q] = q;
        auto tkey = [&](int t) { return std::min({m.tri[3 * (size_t)t], m.tri[3 * (size_t)t + 1], m.tri[3 * (size_t)t + 2]}); };
        auto ekey = [&](int e) { return std::min(m.edge[4 * (size_t)e], m.edge[4 * (size_t)e + 1]); };
        std::stable_sort(tord.begin(), tord.end(), [&](int a, int b) { return tkey(a) < tkey(b); });
        std::stable_sort(eord.begin(), eord.end(), [&](int a, int b) { return ekey(a) < ekey(b); });
        for (int q = 0; q < m.nt; ++q) {
            const int t = tord[q];
            for (int j = 0; j < 3; ++j) tri_p[3 * (size_t)q + j] = m.tri[3 * (size_t)t + j];
            tpos[t] = q;
            At0_p[q] = R(m.At0[t]);
        }
        // triangle of each directed edge: (v0, v1) -> triangle containing it
        std::unordered_map<long long, int> dir_tri;
        dir_tri.reserve(3 * (size_t)m.nt);
        for (int t = 0; t < m.nt; ++t)
            for (int k = 0; k < 3; ++k)
                dir_tri[(long long)m.tri[3 * t + k] * m.nv + m.tri[3 * t + (k + 1) % 3]] = t;
        for (int q = 0; q < m.ne; ++q) {
            const int e = eord[q];
            const int *E = &m.edge[4 * (size_t)e];
            for (int j = 0; j < 4; ++j) edge_p[4 * (size_t)q + j] = E[j];
            etri_p[2 * (size_t)q] = tpos[dir_tri.at((long long)E[0] * m.nv + E[1])];
            etri_p[2 * (size_t)q + 1] = tpos[dir_tri.at((long long)E[1] * m.nv + E[0])];
            invL0[q] = R(1.0 / m.L0[e]);
            th0[q] = R(m.th0[e]);
        }
        // the triangles of each vertex (processing order): {triangle, next
        // corner, the one after}
        std::vector<std::vector<int4>> tris(m.nv);
        std::vector<int4> tri4(m.nt);
        for (int q = 0; q < m.nt; ++q) {
            const int *T = &tri_p[3 * (size_t)q];
            tri4[q] = make_int4(T[0], T[1], T[2], 0);
            for (int r = 0; r < 3; ++r) tris[T[r]].push_back(make_int4(q, T[(r + 1) % 3], T[(r + 2) % 3], 0));
        }
        int maxv = 0;  // largest valence (on a closed manifold: triangles = edges per vertex)
        for (int i = 0; i < m.nv; ++i) maxv = std::max(maxv, (int)tris[i].size());
        // the fan of each vertex i in cyclic order: triangles T_k = (i, j_k,
        // j_k+1) as oriented, so that consecutive T_k share the edge (i, j_k).
        // Slot 0 repeats the last entry (the loop's carried values start
        // from it), slots 1..deg hold k = 0..deg-1; per entry {T_k, j_k,
        // edge (i, j_k) << 1 | role of i in it, edge (j_k, j_k+1)}.
        std::unordered_map<long long, int> pair_edge;
        pair_edge.reserve(2 * (size_t)m.ne);
        for (int q = 0; q < m.ne; ++q) {
            const int a = edge_p[4 * (size_t)q], b = edge_p[4 * (size_t)q + 1];
            pair_edge[(long long)std::min(a, b) * m.nv + std::max(a, b)] = q;
        }
        auto edge_of = [&](int a, int b) { return pair_edge.at((long long)std::min(a, b) * m.nv + std::max(a, b)); };
        std::vector<int4> vfan((size_t)(maxv + 1) * m.nv, make_int4(-1, 0, 0, 0));
        for (int i = 0; i < m.nv; ++i) {
            std::unordered_map<int, int4> from;  // j_k -> {T_k, j_k, j_k+1}
            for (const int4 &g : tris[i]) from[g.y] = make_int4(g.x, g.y, g.z, 0);
            const int deg = (int)tris[i].size();
            std::vector<int4> fan;
            int j = tris[i][0].y;
            for (int k = 0; k < deg; ++k) {
                const auto it = from.find(j);
                if (it == from.end()) return fail(HEMO_ERR_ARG, "mesh: a vertex's triangles do not form one fan");
                const int4 T = it->second;
                const int e = edge_of(i, j), role = edge_p[4 * (size_t)e] == i ? 0 : 1;
                // the edge's triangle lists: (v0, v1, a) first, (v1, v0, b) second
                const int t_in = etri_p[2 * (size_t)e + role];  // contains i -> j
                if (t_in != T.x) return fail(HEMO_ERR_ARG, "mesh: inconsistent orientation in a vertex fan");
                fan.push_back(make_int4(T.x, j, (e << 1) | role, edge_of(T.y, T.z)));
                j = T.z;
            }
            if (j != tris[i][0].y) return fail(HEMO_ERR_ARG, "mesh: a vertex's fan does not close");
            vfan[i] = fan[deg - 1];
            for (int k = 0; k < deg; ++k) vfan[(size_t)(k + 1) * m.nv + i] = fan[k];
        }
        int4 *dvfan = (int4 *)dalloc(s, sizeof(int4) * vfan.size());
        if (!dvfan) return fail(HEMO_ERR_OOM, "device allocation of mesh tables failed");
        HEMO_CU(cudaMemcpy(dvfan, vfan.data(), sizeof(int4) * vfan.size(), cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(dtri4, tri4.data(), sizeof(int4) * tri4.size(), cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(dtri, tri_p.data(), sizeof(int) * tri_p.size(), cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(dedge, edge_p.data(), sizeof(int) * edge_p.size(), cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(detri, etri_p.data(), sizeof(int) * etri_p.size(), cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(dL0, invL0.data(), rs * m.ne, cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(dth0, th0.data(), rs * m.ne, cudaMemcpyHostToDevice));
        MeshDev<R> d{};
        d.nv = m.nv;
        d.nt = m.nt;
        d.ne = m.ne;
        d.tri = dtri;
        d.edge = dedge;
        d.etri = detri;
        d.invL0 = dL0;
        d.th0 = dth0;
        d.tri4 = dtri4;
        d.maxv = maxv;
        d.vfan = dvfan;
        d.tstride = coprime_stride(m.nt);
        d.estride = coprime_stride(m.ne);
        R *dAt0 = (R *)dalloc(s, rs * m.nt);
        if (!dAt0) return fail(HEMO_ERR_OOM, "device allocation of mesh tables failed");
        HEMO_CU(cudaMemcpy(dAt0, At0_p.data(), rs * m.nt, cudaMemcpyHostToDevice));
        d.At0 = dAt0;
        d.k_local = R(m.k_local);
        d.thm2i = m.theta_m > 0 ? R(1.0 / (m.theta_m * m.theta_m)) : R(0);
        d.A0 = m.A0;
        d.V0 = m.V0;
        d.K = R(m.k_link * m.kbt / m.persistence);
        d.m2 = R(m.max_strain * m.max_strain);
        d.kb = R(m.k_bend * m.kbt);
        d.k_area = m.k_area;
        d.k_volume = m.k_volume;
        d.Ku = R(m.kbt / m.persistence);
        d.kbu = R(m.kbt);
        d.k_link = R(m.k_link);
        d.k_bend = R(m.k_bend);
        md[t] = d;
    }
    HEMO_CU(cudaMemcpy(s->meshes_d, md.data(), sizeof(MeshDev<R>) * MAX_TYPES, cudaMemcpyHostToDevice));

    // cells: FP64 centroid (vertex mean) and offsets in R
    if (nc) {
        std::vector<double> ctr(3 * nc, 0.0);
        std::vector<R> off(3 * (size_t)nv);
        for (int c = 0; c < nc; ++c) {
            const int n = s->meshes[s->cell_type[c]].nv, o = s->cell_first[c];
            for (int i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d) ctr[3 * c + d] += s->X0[3 * (size_t)(o + i) + d];
            for (int d = 0; d < 3; ++d) ctr[3 * c + d] /= n;
            for (int i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d)
                    off[3 * (size_t)(o + i) + d] = R(s->X0[3 * (size_t)(o + i) + d] - ctr[3 * c + d]);
        }
        HEMO_CU(cudaMemcpy(s->ctr, ctr.data(), sizeof(double) * 3 * nc, cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(s->off, off.data(), rs * 3 * (size_t)nv, cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(s->vcell_d, s->vcell.data(), sizeof(int) * nv, cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(s->cell_first_d, s->cell_first.data(), sizeof(int) * nc, cudaMemcpyHostToDevice));
        HEMO_CU(cudaMemcpy(s->cell_type_d, s->cell_type.data(), sizeof(int) * nc, cudaMemcpyHostToDevice));
    }
    const size_t smem = cell_smem_bytes<R>(s->max_nv, s->max_nt, s->max_ne);
    if (smem > 48 * 1024) HEMO_CU(set_cell_smem_limit<R>(smem));
    const size_t smem_adj = cell_adjoint_smem_bytes<R>(s->max_nv, s->max_nt);
    if (smem_adj > 48 * 1024) HEMO_CU(set_cell_adjoint_smem_limit<R>(smem_adj));
    if (std::is_same<R, float>::value) {
        const size_t gs = cell_adjoint_gather_bytes(s->max_nv, s->max_nt, s->max_ne);
        if (gs > 48 * 1024 && gs <= CELL_ADJ_GATHER_MAX_SMEM) HEMO_CU(set_cell_adjoint_gather_smem_limit(gs));
    }
    if (!nc) {  // no cells: the force field is the body force, written once
        View<R> v = make_view<R>(s);
        launch_spread<R>(v, st);
    }
    HEMO_CU(cudaGetLastError());
    s->finalized = true;
    return HEMO_OK;
}

int ensure_ready(hemo_sim *s) {
    if (s->finalized) return HEMO_OK;
    return is_f64(s) ? finalize_impl<double>(s) : finalize_impl<float>(s);
}

// The step variant k = parity + 2 force + 4 integ, or 12 + parity + 2 integ
// with the adaptive separation, captured on first use.
template <typename R>
int capture_graph(hemo_sim *s, int k) {
    cudaGraph_t g = nullptr;
    View<R> v = make_view<R>(s);
    const bool adaptive = k >= 12;
    v.integ = adaptive ? (k - 12) >> 1 : k >> 2;
    HEMO_CU(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    enqueue_step<R>(s, v, k & 1, adaptive ? 2 : (k >> 1) & 1, s->cap);
    cudaError_t e = cudaStreamEndCapture(s->cap, &g);
    if (e != cudaSuccess) return fail(HEMO_ERR_CUDA, std::string("step capture: ") + cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int kernels = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
    }
    s->graph_kernels[k] = kernels;
    e = cudaGraphInstantiate(&s->graph[k], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(HEMO_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return HEMO_OK;
}

int poll_status(hemo_sim *s) {
    if (s->ev_pending && cudaEventQuery(s->ev) == cudaSuccess) {
        s->sticky |= *s->status_host;
        s->ev_pending = false;
    }
    cudaGetLastError();
    return status_code(s->sticky);
}

double dihedral(D3 p0, D3 p1, D3 pa, D3 pb) {
    const D3 e = sub(p1, p0);
    const D3 n1 = crs(e, sub(pa, p0)), n2 = crs(sub(pb, p0), e);
    return std::atan2(dt3(crs(n1, n2), e) / std::sqrt(dt3(e, e)), dt3(n1, n2));
}

int copy_out(hemo_sim *s, void *dst, const void *src, size_t bytes) {
    if (!dst || !bytes) return HEMO_OK;
    HEMO_CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s->stream));
    return HEMO_OK;
}

}  // namespace


// ---------------------------------------------------------------------------
// differentiation form: checkpoints, loss, reverse sweep
// ---------------------------------------------------------------------------
namespace {

template <typename A, typename B>
__global__ void convert_kernel(const A *in, B *out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (B)in[i];
}

template <typename A, typename B>
void convert(const A *in, B *out, size_t n, cudaStream_t st) {
    if (n) convert_kernel<A, B><<<(int)((n + 255) / 256), 256, 0, st>>>(in, out, n);
}

size_t lat_bytes(const hemo_sim *s) { return rsize(s) * Q * (size_t)s->N; }

// reference centroids of the loss's drift term := current centroids
template <typename R>
int set_reference_centroids(hemo_sim *s) {
    if (!s->ncell) return HEMO_OK;
    int rc = ensure_staging(s, sizeof(double) * 6 * (size_t)s->ncell);
    if (rc) return rc;
    launch_cell_forces<R>(make_view<R>(s), 1, (double *)s->staging, s->stream);
    std::vector<double> st(6 * (size_t)s->ncell), c0(3 * (size_t)s->ncell);
    HEMO_CU(cudaMemcpyAsync(st.data(), s->staging, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, s->stream));
    HEMO_CU(cudaStreamSynchronize(s->stream));
    for (int c = 0; c < s->ncell; ++c)
        for (int k = 0; k < 3; ++k) c0[3 * c + k] = st[6 * c + k];
    if (!s->c0) s->c0 = (double *)dalloc(s, sizeof(double) * c0.size());
    if (!s->c0) return fail(HEMO_ERR_OOM, "allocation of reference centroids failed");
    HEMO_CU(cudaMemcpy(s->c0, c0.data(), sizeof(double) * c0.size(), cudaMemcpyHostToDevice));
    return HEMO_OK;
}

template <typename R>
int save_checkpoint(hemo_sim *s) {
    const size_t k = (size_t)((s->steps_done - s->rec_start) / s->ck_every);
    while (s->ck_f.size() <= k) {
        void *f = dalloc(s, lat_bytes(s));
        void *c = dalloc(s, sizeof(double) * 3 * std::max(s->ncell, 1));
        void *o = dalloc(s, rsize(s) * 3 * std::max(s->nv, 1));
        if (!f || !c || !o) return fail(HEMO_ERR_OOM, "checkpoint allocation failed");
        s->ck_f.push_back(f);
        s->ck_ctr.push_back(c);
        s->ck_off.push_back(o);
    }
    View<R> v = make_view<R>(s);
    launch_copy_natural<R>(v, s->precision, s->le ? 0 : (int)(s->steps_done & 1), (R *)s->ck_f[k], s->stream);
    HEMO_CU(cudaMemcpyAsync(s->ck_ctr[k], s->ctr, sizeof(double) * 3 * s->ncell, cudaMemcpyDeviceToDevice, s->stream));
    HEMO_CU(cudaMemcpyAsync(s->ck_off[k], s->off, rsize(s) * 3 * s->nv, cudaMemcpyDeviceToDevice, s->stream));
    HEMO_CU(cudaGetLastError());
    return HEMO_OK;
}

void clear_segment_graphs(hemo_sim *s) {
    for (auto &kv : s->seg_graphs) cudaGraphExecDestroy(kv.second);
    s->seg_graphs.clear();
}

void *grow(hemo_sim *s, void *&p, size_t &have, size_t need) {
    if (have >= need && p) return p;
    dfree(s, p);
    p = dalloc(s, need);
    have = p ? need : 0;
    return p;
}

// Enqueues one checkpoint segment of the reverse sweep: forward recomputation
// of `len` steps from the state already restored, each step writing its force
// field, velocity, membrane forces, anchors, bins, re-based offsets and the
// collision density and velocity into the step's own slots, then the adjoint
// steps in reverse.  The adjoint-of-f buffers alternate; `a` holds them in
// the order at entry.
template <typename R>
void enqueue_segment(hemo_sim *s, AdjView<R> a, int len, cudaStream_t st) {
    AdjBuffers &b = s->adj;
    const size_t N = (size_t)s->N, nv = (size_t)s->nv;
    const size_t nb1 = (size_t)s->nbins + 1;
    const View<R> v = make_view<R>(s);
    R *rec = (R *)b.seg_rec;
    auto slot = [&](int j) {  // the quantities of step s0 + j
        View<R> vj = v;
        vj.u = (R *)b.seg_u + 3 * N * j;
        vj.rec = rec + 4 * N * j;
        if (s->ncell) {
            vj.F = (R *)b.seg_F + 3 * N * j;
            vj.Fv = (R *)b.seg_Fv + 3 * nv * j;
            vj.anc_i = (int *)b.seg_anc_i + 3 * nv * j;
            vj.anc_t = (R *)b.seg_anc_t + 3 * nv * j;
            vj.perm = (int *)b.seg_perm + nv * j;
            vj.start = (int *)b.seg_start + nb1 * j;
            vj.off_rec = (R *)b.seg_off + 3 * nv * j;
        }
        return vj;
    };
    for (int j = 0; j < len; ++j) enqueue_step<R>(s, slot(j), j & 1, true, st);
    launch_rho_out<R>(v, s->precision, len & 1, rec + 4 * N * len, st);  // density after the segment
    for (int j = len - 1; j >= 0; --j) {
        View<R> vj = slot(j);
        vj.rec = nullptr;
        vj.off_rec = nullptr;
        vj.off = (R *)b.seg_off + 3 * nv * j;
        a.rec = rec + 4 * N * j;
        a.rho1 = rec + 4 * N * (j + 1);
        a.up = vj.u;
        if (s->ncell) {
            View<R> vl = vj;  // spreading of lamX into lamu at every node
            vl.Fv = a.lamX;
            vl.F = a.lamu;
            vl.g[0] = vl.g[1] = vl.g[2] = R(0);
            vl.spread_all_nodes = 1;
            launch_spread<R>(vl, st);                                       // lamu = S lamX
            launch_vertex_field<R>(vj, a.up, a.lamX, a.lamX, nullptr, st);  // + (u' . lamX) grad w
        } else {
            cudaMemsetAsync(a.lamu, 0, sizeof(R) * 3 * N, st);
        }
        launch_adj_moments<R>(vj, a, st);
        launch_adj_collide<R>(vj, a, st);
        if (s->ncell) {
            launch_vertex_field<R>(vj, a.lamF, vj.Fv, a.lamX, a.lamFv, st);  // lamFv = I lamF; + (F_v . lamF) grad w
            launch_cell_adjoint<R>(vj, a, st);                               // + Hessian lamFv; moduli
        }
        std::swap(a.lamf_in, a.lamf_out);
    }
}

template <typename R>
int backward_impl(hemo_sim *s, const double *dL_dverts, double *grad, int ngrad) {
    const int nt = (int)s->meshes.size();
    const int ng = 4 * nt + 4;
    const long long t_end = s->steps_done;
    const int K = s->ck_every;
    const size_t N = (size_t)s->N, nv = (size_t)s->nv, rs = sizeof(R);
    const size_t nv1 = std::max<size_t>(nv, 1), nc1 = (size_t)std::max(s->ncell, 1), nb1 = (size_t)s->nbins + 1;
    cudaStream_t st = s->stream;
    int rc;
    HEMO_CU(cudaStreamSynchronize(st));
    AdjBuffers &b = s->adj;
    bool moved = false;
    auto need = [&](void *&p, size_t &have, size_t bytes) {
        const void *old = p;
        const bool ok = grow(s, p, have, bytes) != nullptr;
        moved |= p != old;
        return ok;
    };
    if (!need(b.lamf_in, b.sz_lamf_in, rs * Q * N) || !need(b.lamf_out, b.sz_lamf_out, rs * Q * N) ||
        !need(b.lamu, b.sz_lamu, rs * 3 * N) || !need(b.lamF, b.sz_lamF, rs * 3 * N) ||
        !need(b.lamX, b.sz_lamX, rs * 3 * nv1) || !need(b.lamFv, b.sz_lamFv, rs * 3 * nv1) ||
        !need(b.grad, b.sz_grad, sizeof(double) * ng) || !need(b.amom, b.sz_amom, rs * 4 * N) ||
        !need(b.seg_rec, b.sz_seg_rec, rs * 4 * N * (size_t)(K + 1)) ||
        !need(b.seg_F, b.sz_seg_F, rs * 3 * N * (size_t)(s->ncell ? K : 1)) ||
        !need(b.seg_u, b.sz_seg_u, rs * 3 * N * (size_t)K) ||
        !need(b.seg_off, b.sz_seg_off, rs * 3 * nv1 * (size_t)K) ||
        !need(b.seg_Fv, b.sz_seg_Fv, rs * 3 * nv1 * (size_t)K) ||
        !need(b.seg_anc_i, b.sz_seg_anc_i, sizeof(int) * 3 * nv1 * (size_t)K) ||
        !need(b.seg_anc_t, b.sz_seg_anc_t, rs * 3 * nv1 * (size_t)K) ||
        !need(b.seg_perm, b.sz_seg_perm, sizeof(int) * nv1 * (size_t)K) ||
        !need(b.seg_start, b.sz_seg_start, sizeof(int) * nb1 * (size_t)K) ||
        !need(b.fin_f, b.sz_fin_f, rs * Q * N) || !need(b.fin_u, b.sz_fin_u, rs * 3 * N) ||
        !need(b.fin_ctr, b.sz_fin_ctr, sizeof(double) * 3 * nc1) || !need(b.fin_off, b.sz_fin_off, rs * 3 * nv1))
        return fail(HEMO_ERR_OOM, "allocation of adjoint buffers failed");
    if (moved) clear_segment_graphs(s);  // captured pointers are stale
    View<R> v = make_view<R>(s);
    // final state, restored at the end
    launch_copy_natural<R>(v, s->precision, (int)(t_end & 1), (R *)b.fin_f, st);
    HEMO_CU(cudaMemcpyAsync(b.fin_u, s->u, rs * 3 * N, cudaMemcpyDeviceToDevice, st));
    HEMO_CU(cudaMemcpyAsync(b.fin_ctr, s->ctr, sizeof(double) * 3 * s->ncell, cudaMemcpyDeviceToDevice, st));
    HEMO_CU(cudaMemcpyAsync(b.fin_off, s->off, rs * 3 * nv, cudaMemcpyDeviceToDevice, st));
    // adjoint of the final state: dL/dX_T given, dL/df_T = 0
    if (nv) {
        if ((rc = ensure_staging(s, sizeof(double) * 3 * nv))) return rc;
        HEMO_CU(cudaMemcpyAsync(s->staging, dL_dverts, sizeof(double) * 3 * nv, cudaMemcpyDefault, st));
        convert<double, R>((const double *)s->staging, (R *)b.lamX, 3 * nv, st);
    }
    HEMO_CU(cudaMemsetAsync(b.lamf_in, 0, rs * Q * N, st));
    HEMO_CU(cudaMemsetAsync(b.grad, 0, sizeof(double) * ng, st));
    AdjView<R> a{};
    a.lamu = (R *)b.lamu;
    a.lamF = (R *)b.lamF;
    a.amom = (R *)b.amom;
    a.lamX = (R *)b.lamX;
    a.lamFv = (R *)b.lamFv;
    a.grad = (double *)b.grad;
    a.ntypes = nt;
    int in_first = 0;  // which buffer holds the adjoint of f at the current step
    const long long nseg = (t_end - s->rec_start + K - 1) / K;
    for (long long seg = nseg - 1; seg >= 0; --seg) {
        const long long s0 = s->rec_start + seg * K, s1 = std::min<long long>(s0 + K, t_end);
        const int len = (int)(s1 - s0);
        launch_restore_natural<R>(v, s->precision, 0, (const R *)s->ck_f[seg], st);
        HEMO_CU(cudaMemcpyAsync(s->ctr, s->ck_ctr[seg], sizeof(double) * 3 * s->ncell, cudaMemcpyDeviceToDevice, st));
        HEMO_CU(cudaMemcpyAsync(s->off, s->ck_off[seg], rs * 3 * nv, cudaMemcpyDeviceToDevice, st));
        a.lamf_in = (R *)(in_first ? b.lamf_out : b.lamf_in);
        a.lamf_out = (R *)(in_first ? b.lamf_in : b.lamf_out);
        const long long key = 2LL * len + in_first;
        auto it = s->seg_graphs.find(key);
        if (it == s->seg_graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            const bool timing = s->timing;  // no phase-event nodes in the reverse sweep
            s->timing = false;
            HEMO_CU(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
            enqueue_segment<R>(s, a, len, s->cap);
            cudaError_t e = cudaStreamEndCapture(s->cap, &g);
            s->timing = timing;
            if (e != cudaSuccess) return fail(HEMO_ERR_CUDA, std::string("segment capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(HEMO_ERR_CUDA, std::string("segment instantiate: ") + cudaGetErrorString(e));
            it = s->seg_graphs.emplace(key, ge).first;
        }
        HEMO_CU(cudaGraphLaunch(it->second, st));
        if (len & 1) in_first ^= 1;
        s->steps_done = s1;
    }
    // restore the final state
    launch_restore_natural<R>(v, s->precision, (int)(t_end & 1), (const R *)b.fin_f, st);
    HEMO_CU(cudaMemcpyAsync(s->u, b.fin_u, rs * 3 * N, cudaMemcpyDeviceToDevice, st));
    HEMO_CU(cudaMemcpyAsync(s->ctr, b.fin_ctr, sizeof(double) * 3 * s->ncell, cudaMemcpyDeviceToDevice, st));
    HEMO_CU(cudaMemcpyAsync(s->off, b.fin_off, rs * 3 * nv, cudaMemcpyDeviceToDevice, st));
    s->steps_done = t_end;
    std::vector<double> g(ng);
    HEMO_CU(cudaMemcpyAsync(g.data(), b.grad, sizeof(double) * ng, cudaMemcpyDeviceToHost, st));
    HEMO_CU(cudaStreamSynchronize(st));
    HEMO_CU(cudaGetLastError());
    for (int k = 0; k < std::min(ng, ngrad); ++k) grad[k] = g[k];
    return status_code(s->sticky);
}

template <typename R>
int loss_impl(hemo_sim *s, double *loss, double *dL_dverts) {
    const size_t nv = (size_t)s->nv;
    int rc;
    if (!s->c0 && (rc = set_reference_centroids<R>(s))) return rc;
    AdjBuffers &b = s->adj;
    if (!grow(s, b.cell_loss, b.sz_cell_loss, sizeof(double) * std::max(s->ncell, 1)) ||
        !grow(s, b.dldx, b.sz_dldx, sizeof(R) * 3 * std::max<size_t>(nv, 1)))
        return fail(HEMO_ERR_OOM, "allocation of loss buffers failed");
    if ((rc = ensure_staging(s, sizeof(double) * 3 * std::max<size_t>(nv, 1)))) return rc;
    launch_deformation_loss<R>(make_view<R>(s), s->c0, (double *)b.cell_loss, (R *)b.dldx, s->stream);
    std::vector<double> cl(s->ncell);
    HEMO_CU(cudaMemcpyAsync(cl.data(), b.cell_loss, sizeof(double) * cl.size(), cudaMemcpyDeviceToHost, s->stream));
    if (dL_dverts && nv) {
        convert<R, double>((const R *)b.dldx, (double *)s->staging, 3 * nv, s->stream);
        HEMO_CU(cudaMemcpyAsync(dL_dverts, s->staging, sizeof(double) * 3 * nv, cudaMemcpyDefault, s->stream));
    }
    HEMO_CU(cudaStreamSynchronize(s->stream));
    HEMO_CU(cudaGetLastError());
    double L = 0;
    for (double x : cl) L += x;
    if (loss) *loss = s->ncell ? L / s->ncell : 0.0;
    return HEMO_OK;
}

}  // namespace

extern "C" {

int hemo_record(hemo_sim *s, int checkpoint_every) {
    NvtxRange nvtx_("hemo_record");
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if (checkpoint_every < 2 || (checkpoint_every & 1)) return fail(HEMO_ERR_ARG, "checkpoint_every must be even and >= 2");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (s->steps_done & 1) return fail(HEMO_ERR_STATE, "hemo_record: start at an even step count");
    if (s->force_every != 1 || s->integrator != HEMO_EULER || s->force_tol >= 0)
        return fail(HEMO_ERR_STATE, "hemo_record: the differentiation form needs forces every step and Euler");
    for (const HostMesh &m : s->meshes)
        if (m.k_local > 0 || m.theta_m > 0)
            return fail(HEMO_ERR_STATE, "hemo_record: the differentiation form supports the four-term membrane model only");
    if (s->visc_ratio != 1.0) return fail(HEMO_ERR_STATE, "hemo_record: the differentiation form needs a viscosity ratio of 1");
    if (s->le) return fail(HEMO_ERR_STATE, "hemo_record: the differentiation form does not support the Lees-Edwards boundary");
    HEMO_CU(cudaStreamSynchronize(s->stream));
    s->rec = true;
    s->ck_every = checkpoint_every;
    s->rec_start = s->steps_done;
    rc = is_f64(s) ? set_reference_centroids<double>(s) : set_reference_centroids<float>(s);
    if (rc) return rc;
    rc = is_f64(s) ? save_checkpoint<double>(s) : save_checkpoint<float>(s);
    if (rc) return rc;
    HEMO_CU(cudaStreamSynchronize(s->stream));
    return HEMO_OK;
}

int hemo_deformation_loss(hemo_sim *s, double *loss, double *dL_dverts) {
    NvtxRange nvtx_("hemo_deformation_loss");
    if (!s || !loss) return fail(HEMO_ERR_ARG, "null pointer");
    int rc = ensure_ready(s);
    if (rc) return rc;
    return is_f64(s) ? loss_impl<double>(s, loss, dL_dverts) : loss_impl<float>(s, loss, dL_dverts);
}

int hemo_backward(hemo_sim *s, const double *dL_dverts, double *grad, int ngrad) {
    NvtxRange nvtx_("hemo_backward");
    if (!s || !grad || (s->nv && !dL_dverts)) return fail(HEMO_ERR_ARG, "null pointer");
    if (ngrad < 4 * (int)s->meshes.size() + 4) return fail(HEMO_ERR_ARG, "grad needs 4 * mesh types + 4 entries");
    if (!s->rec || s->steps_done <= s->rec_start) return fail(HEMO_ERR_STATE, "hemo_backward: nothing recorded (hemo_record, then hemo_step)");
    int rc = poll_status(s);
    if (rc) return rc;
    return is_f64(s) ? backward_impl<double>(s, dL_dverts, grad, ngrad) : backward_impl<float>(s, dL_dverts, grad, ngrad);
}

}  // extern "C"

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *hemo_last_error(void) { return g_err.c_str(); }

int hemo_velocity_set(int32_t *c, double *w) {
    if (!c || !w) return fail(HEMO_ERR_ARG, "hemo_velocity_set: null pointer");
    for (int i = 0; i < Q; ++i) {
        c[3 * i] = cx(i);
        c[3 * i + 1] = cy(i);
        c[3 * i + 2] = cz(i);
        w[i] = wgt(i);
    }
    return HEMO_OK;
}

// Rows (x-lines, index y + ny z) for the staged collision.  A row is
// interior when it and the eight rows around it (the y-z offsets of D3Q19)
// lie in the lattice, or wrap on periodic axes, and hold fluid only, with x
// periodic: none of its populations meets a wall.  Runs of interior rows
// within a z-plane are cut into tiles of at most tile_rows rows; the rows
// that are not interior but hold fluid go to the per-node kernel.  Staging
// needs 16-byte aligned rows (bulk copies), rows of at most 1024 nodes (a
// stage's range) and at least two stages of the ring in shared memory (one
// CTA per SM takes up to four), and is for 2-byte storage only.  By default
// it is used for rows of at least 512 nodes (measured: on the 1000-node
// rows of the pipe it takes 13 % less time than the per-node kernel, on
// 128-node rows about as long); on request (HEMO_OPT_STAGED_COLLISION) for
// shorter rows too; never with HEMO_OPT_UNSTAGED_COLLISION.
constexpr size_t TILE_RING_BYTES = 227 * 1024;  // the largest dynamic shared memory of a CTA
constexpr int TILE_STAGE_NODES = 1024;          // as the kernel's stage layout
constexpr int TILE_DEFAULT_MIN_NX = 512;

int plan_rows(hemo_sim *s, const uint8_t *mask) {
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const size_t S = tsize(s), Rb = rsize(s);
    if (S != 2 || (s->options & HEMO_OPT_UNSTAGED_COLLISION) || !s->per[0]) return HEMO_OK;
    if (!(s->options & HEMO_OPT_STAGED_COLLISION) && nx < TILE_DEFAULT_MIN_NX) return HEMO_OK;
    if (((size_t)nx * S) % 16 || ((size_t)nx * Rb) % 16) return HEMO_OK;
    if (nx > TILE_STAGE_NODES) return HEMO_OK;
    // whole rows per tile, as many as a stage's ranges hold
    const size_t per_node = Q * S + 3 * Rb;
    const int k = std::min(TILE_STAGE_NODES / nx, ny);
    const size_t stage = (size_t)TILE_STAGE_NODES * per_node;
    const int stages = (int)std::min<size_t>(4, (TILE_RING_BYTES - 128) / stage);
    if (stages < 2) return HEMO_OK;
    std::vector<uint8_t> fluid((size_t)ny * nz, 1), any((size_t)ny * nz, mask ? 0 : 1);
    if (mask)
        for (int r = 0; r < ny * nz; ++r)
            for (int x = 0; x < nx; ++x) {
                const bool fl = mask[(size_t)r * nx + x] == 0;
                fluid[r] &= fl;
                any[r] |= fl;
            }
    auto row_fluid = [&](int y, int z) {
        if (y < 0 || y >= ny) {
            if (!s->per[1]) return false;
            y = (y + ny) % ny;
        }
        if (z < 0 || z >= nz) {
            if (!s->per[2]) return false;
            z = (z + nz) % nz;
        }
        return fluid[(size_t)y + (size_t)ny * z] != 0;
    };
    auto interior = [&](int y, int z) {
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                if (!row_fluid(y + dy, z + dz)) return false;
        return true;
    };
    std::vector<int4> tiles;
    std::vector<int> erows;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny;) {
            if (interior(y, z)) {
                int len = 1;
                while (len < k && y + len < ny && interior(y + len, z)) ++len;
                tiles.push_back(make_int4(y + ny * z, len, y, z));
                y += len;
            } else {
                if (any[(size_t)y + (size_t)ny * z]) erows.push_back(y + ny * z);
                ++y;
            }
        }
    if (tiles.empty()) return HEMO_OK;
    const int nsm = s->nsm;
    const int smem = (int)(128 + stages * stage);
    HEMO_CU(set_tile_smem_limit(s->precision, (int)TILE_RING_BYTES));  // the cap of every plan
    s->rtiles = (int4 *)dalloc(s, sizeof(int4) * tiles.size());
    s->erows = (int *)dalloc(s, sizeof(int) * std::max<size_t>(erows.size(), 1));
    if (!s->rtiles || !s->erows) return fail(HEMO_ERR_OOM, "allocation of the row tables failed");
    HEMO_CU(cudaMemcpyAsync(s->rtiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, s->stream));
    if (!erows.empty())
        HEMO_CU(cudaMemcpyAsync(s->erows, erows.data(), sizeof(int) * erows.size(), cudaMemcpyHostToDevice, s->stream));
    HEMO_CU(cudaStreamSynchronize(s->stream));  // the host vectors go out of scope
    s->ntiles = (int)tiles.size();
    s->nerows = (int)erows.size();
    s->tile_rows = k;
    s->tile_stages = stages;
    s->tile_grid = std::min(s->ntiles, std::max(nsm, 1));  // one persistent CTA per SM
    s->tile_smem = smem;
    return HEMO_OK;
}

int hemo_create_lattice(const hemo_lattice_desc *d, hemo_sim **out) {
    NvtxRange nvtx_("hemo_create_lattice");
    if (!d || !out) return fail(HEMO_ERR_ARG, "hemo_create_lattice: null pointer");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(HEMO_ERR_ARG, "lattice sizes must be >= 1");
    const long long N = (long long)d->nx * d->ny * d->nz;
    if (N > 0x7fffffffLL / 2) return fail(HEMO_ERR_ARG, "lattice too large (2^30 nodes or more)");
    if (!(d->tau > 0.5)) return fail(HEMO_ERR_ARG, "tau must exceed 1/2");
    if (d->precision < HEMO_F64 || d->precision > HEMO_BF16DEV) return fail(HEMO_ERR_ARG, "unknown precision");
    for (int k = 0; k < 3; ++k)
        if (d->periodic[k] != 0 && d->periodic[k] != 1) return fail(HEMO_ERR_ARG, "periodic flags must be 0 or 1");
    if ((d->alloc == nullptr) != (d->release == nullptr)) return fail(HEMO_ERR_ARG, "alloc and release must be given together");
    bool walls = false;
    if (d->wall_mask)
        for (long long n = 0; n < N; ++n) {
            if (d->wall_mask[n] > 3) return fail(HEMO_ERR_ARG, "wall mask values must be 0..3");
            walls |= d->wall_mask[n] != 0;
        }

    hemo_sim *s = new hemo_sim();
    s->has_walls = walls;
    s->precision = d->precision;
    s->nx = d->nx;
    s->ny = d->ny;
    s->nz = d->nz;
    s->N = N;
    for (int k = 0; k < 3; ++k) {
        s->per[k] = d->periodic[k];
        s->g[k] = d->body_force[k];
        s->uw[0][k] = d->wall_velocity[0][k];
        s->uw[1][k] = d->wall_velocity[1][k];
    }
    s->tau = d->tau;
    s->options = d->options;
    s->stream = (cudaStream_t)d->cuda_stream;
    s->alloc = d->alloc;
    s->release = d->release;
    s->ctx = d->alloc_ctx;
    s->nb[0] = (s->nx + BLK - 1) / BLK;
    s->nb[1] = (s->ny + BLK - 1) / BLK;
    s->nb[2] = (s->nz + BLK - 1) / BLK;
    s->nbins = s->nb[0] * s->nb[1] * s->nb[2];

    auto bail = [&](int code) {
        hemo_destroy(s);
        return code;
    };
    s->f = dalloc(s, tsize(s) * Q * (size_t)N);
    s->ntype = (uint8_t *)dalloc(s, (size_t)N);
    s->links = (uint64_t *)dalloc(s, 8 * (size_t)N);
    s->F = dalloc(s, rsize(s) * 3 * (size_t)N);
    s->u = dalloc(s, rsize(s) * 3 * (size_t)N);
    s->status = (unsigned *)dalloc(s, sizeof(unsigned));
    if (tsize(s) == 2) s->rref = (float2 *)dalloc(s, sizeof(float2) * (size_t)s->ny * s->nz);
    if (!s->f || !s->ntype || !s->links || !s->F || !s->u || !s->status || (tsize(s) == 2 && !s->rref))
        return bail(fail(HEMO_ERR_OOM, "device allocation of the lattice failed"));
    if (s->rref && cudaMemsetAsync(s->rref, 0, sizeof(float2) * (size_t)s->ny * s->nz, s->stream) != cudaSuccess)
        return bail(fail(HEMO_ERR_CUDA, "memset failed"));
    s->u_tma = encode_u_tmap(s);
    if (cudaHostAlloc((void **)&s->status_host, sizeof(unsigned), cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(HEMO_ERR_CUDA, std::string("stream/event setup: ") + cudaGetErrorString(cudaGetLastError())));
    *s->status_host = 0;
    cudaStream_t st = s->stream;
    if (cudaMemsetAsync(s->status, 0, sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(s->F, 0, rsize(s) * 3 * (size_t)N, st) != cudaSuccess)
        return bail(fail(HEMO_ERR_CUDA, "memset failed"));
    cudaError_t e = d->wall_mask ? cudaMemcpyAsync(s->ntype, d->wall_mask, (size_t)N, cudaMemcpyHostToDevice, st)
                                 : cudaMemsetAsync(s->ntype, 0, (size_t)N, st);
    if (e != cudaSuccess) return bail(fail(HEMO_ERR_CUDA, std::string("wall mask upload: ") + cudaGetErrorString(e)));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(fail(HEMO_ERR_CUDA, "device query failed"));
    launch_build_links(s->nx, s->ny, s->nz, s->per, s->ntype, s->links, st);
    if (int rc = plan_rows(s, d->wall_mask)) return bail(rc);
    if (is_f64(s)) launch_init_equilibrium<double>(make_view<double>(s), s->precision, nullptr, st);
    else launch_init_equilibrium<float>(make_view<float>(s), s->precision, nullptr, st);
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bail(fail(HEMO_ERR_CUDA, std::string("lattice setup: ") + cudaGetErrorString(e)));
    *out = s;
    return HEMO_OK;
}

int hemo_set_velocity(hemo_sim *s, const double *u) {
    NvtxRange nvtx_("hemo_set_velocity");
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if (s->steps_done) return fail(HEMO_ERR_STATE, "hemo_set_velocity: only before the first step");
    const double *ud = nullptr;
    if (u) {
        int rc = ensure_staging(s, sizeof(double) * 3 * (size_t)s->N);
        if (rc) return rc;
        HEMO_CU(cudaMemcpyAsync(s->staging, u, sizeof(double) * 3 * (size_t)s->N, cudaMemcpyDefault, s->stream));
        ud = (const double *)s->staging;
    }
    if (s->rref && !s->le) {  // 16-bit storage: the rows' mean x-velocity becomes the reference
        if (ud) launch_row_reference(make_view<float>(s), ud, s->rref, s->stream);
        else HEMO_CU(cudaMemsetAsync(s->rref, 0, sizeof(float2) * (size_t)s->ny * s->nz, s->stream));
    }
    if (is_f64(s)) launch_init_equilibrium<double>(make_view<double>(s), s->precision, ud, s->stream);
    else launch_init_equilibrium<float>(make_view<float>(s), s->precision, ud, s->stream);
    HEMO_CU(cudaGetLastError());
    HEMO_CU(cudaStreamSynchronize(s->stream));
    return HEMO_OK;
}

int hemo_add_cells(hemo_sim *s, const hemo_mesh_desc *m, int ncells, const double *centers, const double *rot,
                   int *first_cell_id) {
    NvtxRange nvtx_("hemo_add_cells");
    if (!s || !m) return fail(HEMO_ERR_ARG, "hemo_add_cells: null pointer");
    if (s->finalized || s->steps_done) return fail(HEMO_ERR_STATE, "hemo_add_cells: only before the first step");
    if (s->meshes.size() >= (size_t)MAX_TYPES) return fail(HEMO_ERR_ARG, "too many mesh types");
    if (m->nv < 4 || m->nt < 4 || !m->tri || !m->rest_xyz) return fail(HEMO_ERR_ARG, "mesh needs >= 4 vertices and triangles");
    if (ncells < 0 || (ncells > 0 && (!centers || !rot))) return fail(HEMO_ERR_ARG, "bad cell placement arguments");
    if ((long long)s->nv + (long long)ncells * m->nv > 0x3fffffffLL) return fail(HEMO_ERR_ARG, "too many vertices");
    if (!(m->persistence > 0) || !(m->max_strain > 0) || !(m->kbt >= 0) || !(m->k_local >= 0) || !(m->theta_m >= 0))
        return fail(HEMO_ERR_ARG, "bad membrane parameters");
    HostMesh hm;
    hm.nv = m->nv;
    hm.nt = m->nt;
    hm.tri.assign(m->tri, m->tri + 3 * (size_t)m->nt);
    for (int x : hm.tri)
        if (x < 0 || x >= m->nv) return fail(HEMO_ERR_ARG, "triangle index out of range");
    if (!build_edge_table(m->nv, hm.tri, hm.edge))
        return fail(HEMO_ERR_ARG, "mesh is not a closed, consistently oriented 2-manifold");
    hm.ne = (int)hm.edge.size() / 4;
    const double *r = m->rest_xyz;
    auto P = [&](int i) { return D3{r[3 * i], r[3 * i + 1], r[3 * i + 2]}; };
    hm.L0.resize(hm.ne);
    hm.th0.resize(hm.ne);
    for (int e = 0; e < hm.ne; ++e) {
        const int *E = &hm.edge[4 * e];
        const D3 d = sub(P(E[1]), P(E[0]));
        hm.L0[e] = std::sqrt(dt3(d, d));
        hm.th0[e] = dihedral(P(E[0]), P(E[1]), P(E[2]), P(E[3]));
        if (!(hm.L0[e] > 0)) return fail(HEMO_ERR_ARG, "zero-length rest edge");
    }
    D3 c{0, 0, 0};
    for (int i = 0; i < hm.nv; ++i) {
        c.x += r[3 * i];
        c.y += r[3 * i + 1];
        c.z += r[3 * i + 2];
    }
    c = {c.x / hm.nv, c.y / hm.nv, c.z / hm.nv};
    double A = 0, V = 0;
    hm.At0.resize(hm.nt);
    for (int t = 0; t < hm.nt; ++t) {
        const D3 p0 = P(hm.tri[3 * t]), p1 = P(hm.tri[3 * t + 1]), p2 = P(hm.tri[3 * t + 2]);
        const D3 n = crs(sub(p1, p0), sub(p2, p0));
        hm.At0[t] = 0.5 * std::sqrt(dt3(n, n));
        if (m->k_local > 0 && !(hm.At0[t] > 0)) return fail(HEMO_ERR_ARG, "zero-area rest triangle");
        A += hm.At0[t];
        V += dt3(sub(p0, c), crs(sub(p1, c), sub(p2, c))) / 6.0;
    }
    hm.A0 = A;
    hm.V0 = V;
    if (!(A > 0) || !(V > 0)) return fail(HEMO_ERR_ARG, "rest shape has non-positive area or volume (check orientation)");
    hm.k_link = m->k_link;
    hm.k_bend = m->k_bend;
    hm.k_area = m->k_area;
    hm.k_volume = m->k_volume;
    hm.kbt = m->kbt;
    hm.persistence = m->persistence;
    hm.max_strain = m->max_strain;
    hm.k_local = m->k_local;
    hm.theta_m = m->theta_m;
    const int type = (int)s->meshes.size();
    s->meshes.push_back(hm);
    s->max_nv = std::max(s->max_nv, hm.nv);
    s->max_nt = std::max(s->max_nt, hm.nt);
    s->max_ne = std::max(s->max_ne, hm.ne);
    if (first_cell_id) *first_cell_id = s->ncell;
    for (int k = 0; k < ncells; ++k) {
        const double *R = rot + 9 * (size_t)k;
        const double *C = centers + 3 * (size_t)k;
        s->cell_type.push_back(type);
        s->cell_first.push_back(s->nv);
        for (int i = 0; i < hm.nv; ++i) {
            for (int d = 0; d < 3; ++d)
                s->X0.push_back(C[d] + R[3 * d] * r[3 * i] + R[3 * d + 1] * r[3 * i + 1] + R[3 * d + 2] * r[3 * i + 2]);
            s->vcell.push_back(s->ncell);
        }
        s->nv += hm.nv;
        s->ncell += 1;
    }
    return HEMO_OK;
}

// the adaptive separation evaluates the forces on the next step again
static int adapt_restart(hemo_sim *s) {
    if (!s->adapt) return HEMO_OK;
    const unsigned long long init[4] = {0ull, 0ull, 0ull, 1ull};
    HEMO_CU(cudaMemcpyAsync(s->adapt, init, sizeof init, cudaMemcpyHostToDevice, s->stream));
    HEMO_CU(cudaStreamSynchronize(s->stream));  // (init is on the stack)
    return HEMO_OK;
}

int hemo_step(hemo_sim *s, int nsteps) {
    NvtxRange nvtx_("hemo_step");
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if (nsteps < 0) return fail(HEMO_ERR_ARG, "nsteps must be >= 0");
    int rc = ensure_ready(s);
    if (rc) return rc;
    rc = poll_status(s);
    if (rc) return rc;
    if (nsteps == 0) return HEMO_OK;
    for (int k = 0; k < nsteps; ++k) {
        const bool force = (s->steps_done - s->ts_origin) % s->force_every == 0;
        if (force && s->force_tol < 0) ++s->evals_host;
        const int integ = s->integrator == HEMO_AB2 ? (s->have_prev ? 2 : 1) : 0;
        const int parity = (int)(s->steps_done & 1);
        const int gi = s->force_tol >= 0 ? 12 + parity + 2 * integ : parity + 2 * (int)force + 4 * integ;
        if (!s->graph[gi]) {
            rc = is_f64(s) ? capture_graph<double>(s, gi) : capture_graph<float>(s, gi);
            if (rc) return rc;
        }
        HEMO_CU(cudaGraphLaunch(s->graph[gi], s->stream));
        s->last_graph = gi;
        s->have_prev = s->integrator == HEMO_AB2;
        ++s->steps_done;
        if (s->rec && (s->steps_done - s->rec_start) % s->ck_every == 0) {
            rc = is_f64(s) ? save_checkpoint<double>(s) : save_checkpoint<float>(s);
            if (rc) return rc;
        }
    }
    HEMO_CU(cudaMemcpyAsync(s->status_host, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    HEMO_CU(cudaEventRecord(s->ev, s->stream));
    s->ev_pending = true;
    return HEMO_OK;
}

int hemo_set_time_scales(hemo_sim *s, int force_every, int integrator) {
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if (force_every < 1) return fail(HEMO_ERR_ARG, "force_every must be >= 1");
    if (integrator != HEMO_EULER && integrator != HEMO_AB2) return fail(HEMO_ERR_ARG, "integrator must be HEMO_EULER or HEMO_AB2");
    if (s->rec) return fail(HEMO_ERR_STATE, "hemo_set_time_scales: not while recording for the reverse sweep");
    if (s->le && (force_every != 1 || integrator != HEMO_EULER))
        return fail(HEMO_ERR_STATE, "hemo_set_time_scales: the Lees-Edwards boundary supports forces every step with Euler only");
    s->force_every = force_every;
    s->integrator = integrator;
    s->ts_origin = s->steps_done;
    s->have_prev = false;
    return adapt_restart(s);
}

int hemo_set_force_tolerance(hemo_sim *s, double delta) {
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if (std::isnan(delta)) return fail(HEMO_ERR_ARG, "hemo_set_force_tolerance: delta is NaN");
    if (s->rec) return fail(HEMO_ERR_STATE, "hemo_set_force_tolerance: not while recording for the reverse sweep");
    if (s->le && delta >= 0) return fail(HEMO_ERR_STATE, "hemo_set_force_tolerance: not with the Lees-Edwards boundary");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (delta >= 0 && !s->adapt) {
        s->off_eval = dalloc(s, rsize(s) * 3 * (size_t)std::max(s->nv, 1));
        s->adapt = (unsigned long long *)dalloc(s, ADAPT_WORDS * sizeof(unsigned long long));
        if (!s->off_eval || !s->adapt) return fail(HEMO_ERR_OOM, "adaptive separation buffers");
        HEMO_CU(cudaMemsetAsync(s->adapt, 0, ADAPT_WORDS * sizeof(unsigned long long), s->stream));
    }
    s->force_tol = delta < 0 ? -1.0 : delta;
    s->ts_origin = s->steps_done;
    return adapt_restart(s);
}

int hemo_get_force_evaluations(hemo_sim *s, long long *count) {
    if (!s || !count) return fail(HEMO_ERR_ARG, "null argument");
    long long n = s->evals_host;
    if (s->adapt) {
        unsigned long long d = 0;
        HEMO_CU(cudaMemcpyAsync(&d, s->adapt + 4, sizeof d, cudaMemcpyDeviceToHost, s->stream));
        HEMO_CU(cudaStreamSynchronize(s->stream));
        n += (long long)d;
    }
    *count = n;
    return HEMO_OK;
}

int hemo_set_viscosity_ratio(hemo_sim *s, double ratio) {
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if (!(ratio > 0) || !std::isfinite(ratio)) return fail(HEMO_ERR_ARG, "viscosity ratio must be finite and > 0");
    if (!(0.5 + ratio * (s->tau - 0.5) > 0.5)) return fail(HEMO_ERR_ARG, "viscosity ratio gives tau_in <= 1/2");
    if (s->rec) return fail(HEMO_ERR_STATE, "hemo_set_viscosity_ratio: not while recording for the reverse sweep");
    if (s->le && ratio != 1.0)  // the indicator's z-rays would cross the displaced plane
        return fail(HEMO_ERR_STATE, "hemo_set_viscosity_ratio: not with the Lees-Edwards boundary");
    HEMO_CU(cudaStreamSynchronize(s->stream));
    if (ratio != 1.0 && !s->ind) {
        s->ind = (uint8_t *)dalloc(s, (size_t)s->N);
        s->tog = (int *)dalloc(s, sizeof(int) * (size_t)s->N);
        if (!s->ind || !s->tog) return fail(HEMO_ERR_OOM, "indicator allocation failed");
        HEMO_CU(cudaMemsetAsync(s->tog, 0, sizeof(int) * (size_t)s->N, s->stream));
        HEMO_CU(cudaMemsetAsync(s->ind, 0, (size_t)s->N, s->stream));
    }
    s->visc_ratio = ratio;
    for (int k = 0; k < hemo_sim::NGRAPH; ++k)  // the step graphs carry the relaxation rates
        if (s->graph[k]) {
            cudaGraphExecDestroy(s->graph[k]);
            s->graph[k] = nullptr;
        }
    s->last_graph = -1;
    return HEMO_OK;
}

int hemo_set_lees_edwards(hemo_sim *s, double U) {
    NvtxRange nvtx_("hemo_set_lees_edwards");
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if (!std::isfinite(U) || !(std::fabs(U) < 0.3)) return fail(HEMO_ERR_ARG, "Lees-Edwards velocity must be finite and below 0.3 in magnitude");
    if (s->steps_done || s->le) return fail(HEMO_ERR_STATE, "hemo_set_lees_edwards: only once, before the first step");
    if (!s->per[0] || !s->per[1] || !s->per[2] || s->has_walls)
        return fail(HEMO_ERR_ARG, "hemo_set_lees_edwards: needs a lattice periodic on every axis without walls");
    if (s->force_every != 1 || s->integrator != HEMO_EULER || s->force_tol >= 0)
        return fail(HEMO_ERR_STATE, "hemo_set_lees_edwards: needs forces every step with Euler (hemo_set_time_scales, hemo_set_force_tolerance)");
    if (s->rec) return fail(HEMO_ERR_STATE, "hemo_set_lees_edwards: not while recording");
    if (s->visc_ratio != 1.0) return fail(HEMO_ERR_STATE, "hemo_set_lees_edwards: not with an internal viscosity ratio other than 1");
    s->f2 = dalloc(s, tsize(s) * Q * (size_t)s->N);
    s->le_aux = dalloc(s, rsize(s) * 4 * 2 * (size_t)s->nx * s->ny);
    s->le_n = (long long *)dalloc(s, sizeof(long long));
    if (!s->f2 || !s->le_aux || !s->le_n) return fail(HEMO_ERR_OOM, "Lees-Edwards buffers");
    HEMO_CU(cudaMemsetAsync(s->le_n, 0, sizeof(long long), s->stream));
    if (s->rref) {  // the two-array kernels store plain deviations: re-store without the reference
        launch_reencode(make_view<float>(s), s->precision, s->rref, nullptr, s->stream);
        HEMO_CU(cudaMemsetAsync(s->rref, 0, sizeof(float2) * (size_t)s->ny * s->nz, s->stream));
    }
    s->le = true;
    s->le_U = U;
    for (int k = 0; k < hemo_sim::NGRAPH; ++k)
        if (s->graph[k]) {
            cudaGraphExecDestroy(s->graph[k]);
            s->graph[k] = nullptr;
        }
    s->last_graph = -1;
    return hemo_sync(s);
}

int hemo_get_inside(hemo_sim *s, uint8_t *inside) {
    NvtxRange nvtx_("hemo_get_inside");
    if (!s || !inside) return fail(HEMO_ERR_ARG, "null pointer");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (!s->tog) {
        s->ind = (uint8_t *)dalloc(s, (size_t)s->N);
        s->tog = (int *)dalloc(s, sizeof(int) * (size_t)s->N);
        if (!s->ind || !s->tog) return fail(HEMO_ERR_OOM, "indicator allocation failed");
        HEMO_CU(cudaMemsetAsync(s->tog, 0, sizeof(int) * (size_t)s->N, s->stream));
    }
    if (is_f64(s)) {
        View<double> v = make_view<double>(s);
        v.ind = s->ind;
        v.tog = s->tog;
        launch_inside<double>(v, s->stream);
    } else {
        View<float> v = make_view<float>(s);
        v.ind = s->ind;
        v.tog = s->tog;
        launch_inside<float>(v, s->stream);
    }
    HEMO_CU(cudaGetLastError());
    HEMO_CU(cudaMemcpyAsync(inside, s->ind, (size_t)s->N, cudaMemcpyDefault, s->stream));
    return hemo_sync(s);
}

int hemo_sync(hemo_sim *s) {
    NvtxRange nvtx_("hemo_sync");
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    HEMO_CU(cudaStreamSynchronize(s->stream));
    unsigned st = 0;
    HEMO_CU(cudaMemcpy(&st, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    s->sticky |= st;
    s->ev_pending = false;
    return status_code(s->sticky);
}

int hemo_get_sizes(const hemo_sim *s, long long *n_nodes, long long *n_vertices, int *n_cells, int *n_bins) {
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if (n_nodes) *n_nodes = s->N;
    if (n_vertices) *n_vertices = s->nv;
    if (n_cells) *n_cells = s->ncell;
    if (n_bins) *n_bins = s->nbins;
    return HEMO_OK;
}

int hemo_get_lattice_plan(const hemo_sim *s, int *plan) {
    if (!s || !plan) return fail(HEMO_ERR_ARG, "null pointer");
    plan[0] = s->ntiles;
    plan[1] = s->ntiles ? s->nerows : 0;
    plan[2] = s->tile_rows;
    plan[3] = s->tile_stages;
    return HEMO_OK;
}

int hemo_get_fields(hemo_sim *s, unsigned what, void *rho, void *u, double *verts, double *forces,
                    double *cellstats) {
    NvtxRange nvtx_("hemo_get_fields");
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    int rc = ensure_ready(s);
    if (rc) return rc;
    const size_t N = (size_t)s->N, rs = rsize(s);
    const int layout = s->le ? 0 : (int)(s->steps_done & 1);  // (two-array streaming: natural order)
    size_t need = std::max<size_t>({rs * 3 * N, sizeof(double) * 6 * (size_t)std::max(s->nv, 1),
                                    sizeof(double) * 6 * (size_t)std::max(s->ncell, 1)});
    rc = ensure_staging(s, need);
    if (rc) return rc;
    cudaStream_t st = s->stream;
    if ((what & HEMO_RHO) && rho) {
        if (is_f64(s)) launch_rho_out<double>(make_view<double>(s), s->precision, layout, (double *)s->staging, st);
        else launch_rho_out<float>(make_view<float>(s), s->precision, layout, (float *)s->staging, st);
        if ((rc = copy_out(s, rho, s->staging, rs * N))) return rc;
    }
    if ((what & HEMO_U) && u) {
        if (is_f64(s)) launch_u_out<double>(make_view<double>(s), (double *)s->staging, st);
        else launch_u_out<float>(make_view<float>(s), (float *)s->staging, st);
        if ((rc = copy_out(s, u, s->staging, rs * 3 * N))) return rc;
    }
    if (((what & HEMO_VERTS) && verts) || ((what & HEMO_FORCES) && forces)) {
        double *X = (double *)s->staging, *Fo = X + 3 * (size_t)s->nv;
        if (is_f64(s)) launch_verts_out<double>(make_view<double>(s), X, Fo, st);
        else launch_verts_out<float>(make_view<float>(s), X, Fo, st);
        if ((what & HEMO_VERTS) && (rc = copy_out(s, verts, X, sizeof(double) * 3 * s->nv))) return rc;
        if ((what & HEMO_FORCES) && (rc = copy_out(s, forces, Fo, sizeof(double) * 3 * s->nv))) return rc;
    }
    if ((what & HEMO_CELLSTATS) && cellstats && s->ncell) {
        if (is_f64(s)) launch_cell_forces<double>(make_view<double>(s), 1, (double *)s->staging, st);
        else launch_cell_forces<float>(make_view<float>(s), 1, (double *)s->staging, st);
        if ((rc = copy_out(s, cellstats, s->staging, sizeof(double) * 6 * s->ncell))) return rc;
    }
    HEMO_CU(cudaGetLastError());
    return hemo_sync(s);
}

int hemo_get_populations(hemo_sim *s, double *f) {
    NvtxRange nvtx_("hemo_get_populations");
    if (!s || !f) return fail(HEMO_ERR_ARG, "null pointer");
    int rc = ensure_ready(s);
    if (rc) return rc;
    rc = ensure_staging(s, sizeof(double) * Q * (size_t)s->N);
    if (rc) return rc;
    const int layout = s->le ? 0 : (int)(s->steps_done & 1);  // (two-array streaming: natural order)
    if (is_f64(s)) launch_populations_out<double>(make_view<double>(s), s->precision, layout, (double *)s->staging, s->stream);
    else launch_populations_out<float>(make_view<float>(s), s->precision, layout, (double *)s->staging, s->stream);
    HEMO_CU(cudaGetLastError());
    if ((rc = copy_out(s, f, s->staging, sizeof(double) * Q * (size_t)s->N))) return rc;
    return hemo_sync(s);
}

// ---------------------------------------------------------------------------
// Checkpoint and resume (Sec. 2.6: the simulation is paused, its state kept
// and the run continued).  The state is what changes from step to step; it
// is written as a header followed by the raw device buffers, so a resumed
// run continues with the same bits.
// ---------------------------------------------------------------------------
namespace {

struct StateHeader {
    uint64_t magic;          // STATE_MAGIC
    int64_t N, nv, ncell, precision, le;
    int64_t steps_done, ts_origin;
    int64_t force_every, integrator, have_prev;
    int64_t evals_host;      // force evaluations of constant-schedule steps
    double force_tol;        // adaptive separation (< 0: off)
    int64_t sections;        // number of buffers that follow
};
constexpr uint64_t STATE_MAGIC = 0x324154534f4d4548ull;  // the bytes "HEMOSTA2" in little-endian order

// the buffers of the dynamic state, in order: (device pointer, bytes)
std::vector<std::pair<void *, size_t>> state_sections(hemo_sim *s) {
    const size_t rs = rsize(s), nv = (size_t)s->nv, nc = (size_t)s->ncell;
    std::vector<std::pair<void *, size_t>> v;
    v.push_back({s->f, tsize(s) * Q * (size_t)s->N});   // populations in the in-place layout of the step parity
    v.push_back({s->u, rs * 3 * (size_t)s->N});         // velocity of the last step
    if (s->rref) v.push_back({s->rref, sizeof(float2) * (size_t)s->ny * s->nz});  // 16-bit: the reference they are stored against
    if (nc) {
        v.push_back({s->ctr, sizeof(double) * 3 * nc});  // FP64 centroids
        v.push_back({s->csp, rs * 6 * nc});             // centroid of the last re-base (held-force steps)
        v.push_back({s->off, rs * 3 * nv});             // vertex offsets
        v.push_back({s->Fv, rs * 3 * nv});              // membrane forces (held between evaluations)
        v.push_back({s->Uprev, rs * 3 * nv});           // previous vertex velocity (Adams-Bashforth)
    }
    if (s->le) v.push_back({s->le_n, sizeof(long long)});  // Lees-Edwards step counter
    if (s->force_tol >= 0) {  // adaptive separation: offsets at the last evaluation, decision words
        v.push_back({s->off_eval, rs * 3 * (size_t)std::max(s->nv, 1)});
        v.push_back({s->adapt, ADAPT_WORDS * sizeof(unsigned long long)});
    }
    return v;
}

size_t state_size(hemo_sim *s) {
    size_t b = sizeof(StateHeader);
    for (auto &x : state_sections(s)) b += x.second;
    return b;
}

int state_ready(hemo_sim *s, const char *who) {
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (s->rec) return fail(HEMO_ERR_STATE, std::string(who) + ": not while recording for the reverse sweep");
    return HEMO_OK;
}

}  // namespace

int hemo_state_bytes(hemo_sim *s, size_t *bytes) {
    if (!bytes) return fail(HEMO_ERR_ARG, "hemo_state_bytes: null pointer");
    int rc = state_ready(s, "hemo_state_bytes");
    if (rc) return rc;
    *bytes = state_size(s);
    return HEMO_OK;
}

int hemo_save_state(hemo_sim *s, void *buf, size_t bytes) {
    NvtxRange nvtx_("hemo_save_state");
    int rc = state_ready(s, "hemo_save_state");
    if (rc) return rc;
    if (!buf) return fail(HEMO_ERR_ARG, "hemo_save_state: null buffer");
    if (bytes < state_size(s)) return fail(HEMO_ERR_ARG, "hemo_save_state: buffer smaller than hemo_state_bytes");
    StateHeader h{};
    h.magic = STATE_MAGIC;
    h.N = s->N;
    h.nv = s->nv;
    h.ncell = s->ncell;
    h.precision = s->precision;
    h.le = s->le;
    h.steps_done = s->steps_done;
    h.ts_origin = s->ts_origin;
    h.evals_host = s->evals_host;
    h.force_every = s->force_every;
    h.integrator = s->integrator;
    h.have_prev = s->have_prev;
    h.force_tol = s->force_tol;
    const auto sec = state_sections(s);
    h.sections = (int64_t)sec.size();
    HEMO_CU(cudaMemcpyAsync(buf, &h, sizeof h, cudaMemcpyDefault, s->stream));
    char *p = (char *)buf + sizeof h;
    for (auto &x : sec) {
        HEMO_CU(cudaMemcpyAsync(p, x.first, x.second, cudaMemcpyDefault, s->stream));
        p += x.second;
    }
    return hemo_sync(s);  // (the header is read from the stack before returning)
}

int hemo_load_state(hemo_sim *s, const void *buf, size_t bytes) {
    NvtxRange nvtx_("hemo_load_state");
    int rc = state_ready(s, "hemo_load_state");
    if (rc) return rc;
    if (!buf) return fail(HEMO_ERR_ARG, "hemo_load_state: null buffer");
    if (bytes < sizeof(StateHeader)) return fail(HEMO_ERR_ARG, "hemo_load_state: buffer too small");
    StateHeader h{};
    HEMO_CU(cudaMemcpy(&h, buf, sizeof h, cudaMemcpyDefault));
    if (h.magic != STATE_MAGIC) return fail(HEMO_ERR_ARG, "hemo_load_state: not a saved state");
    if (h.N != s->N || h.nv != s->nv || h.ncell != s->ncell || h.precision != s->precision || h.le != (int64_t)s->le)
        return fail(HEMO_ERR_ARG, "hemo_load_state: the state belongs to a simulation of other sizes, precision or boundary");
    if (h.force_every < 1 || (h.integrator != HEMO_EULER && h.integrator != HEMO_AB2) || h.steps_done < 0 ||
        std::isnan(h.force_tol))
        return fail(HEMO_ERR_ARG, "hemo_load_state: corrupt header");
    if (h.force_tol >= 0) {  // the adaptive separation's buffers, then its state
        if ((rc = hemo_set_force_tolerance(s, h.force_tol))) return rc;
    } else {
        s->force_tol = -1.0;
    }
    const auto sec = state_sections(s);
    if (h.sections != (int64_t)sec.size() || bytes < state_size(s))
        return fail(HEMO_ERR_ARG, "hemo_load_state: buffer size does not match the simulation");
    const char *p = (const char *)buf + sizeof h;
    for (auto &x : sec) {
        HEMO_CU(cudaMemcpyAsync(x.first, p, x.second, cudaMemcpyDefault, s->stream));
        p += x.second;
    }
    s->steps_done = h.steps_done;
    s->ts_origin = h.ts_origin;
    s->evals_host = h.evals_host;
    s->force_every = (int)h.force_every;
    s->integrator = (int)h.integrator;
    s->have_prev = h.have_prev != 0;
    return hemo_sync(s);
}

int hemo_get_links(hemo_sim *s, uint64_t *links) {
    if (!s || !links) return fail(HEMO_ERR_ARG, "null pointer");
    int rc = copy_out(s, links, s->links, 8 * (size_t)s->N);
    if (rc) return rc;
    return hemo_sync(s);
}

int hemo_get_edges(hemo_sim *s, int type, int32_t *edges, int *ne) {
    if (!s || !edges || !ne) return fail(HEMO_ERR_ARG, "null pointer");
    if (type < 0 || type >= (int)s->meshes.size()) return fail(HEMO_ERR_ARG, "no such mesh type");
    const HostMesh &m = s->meshes[type];
    std::memcpy(edges, m.edge.data(), sizeof(int) * m.edge.size());
    *ne = m.ne;
    return HEMO_OK;
}

int hemo_set_vertices(hemo_sim *s, const double *verts) {
    NvtxRange nvtx_("hemo_set_vertices");
    if (!s || !verts) return fail(HEMO_ERR_ARG, "null pointer");
    if (s->steps_done) return fail(HEMO_ERR_STATE, "hemo_set_vertices: only before the first step");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (!s->nv) return HEMO_OK;
    std::vector<double> X(3 * (size_t)s->nv);
    HEMO_CU(cudaMemcpy(X.data(), verts, sizeof(double) * X.size(), cudaMemcpyDefault));
    std::vector<double> ctr(3 * s->ncell, 0.0);
    for (int c = 0; c < s->ncell; ++c) {
        const int n = s->meshes[s->cell_type[c]].nv, o = s->cell_first[c];
        for (int i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) ctr[3 * c + d] += X[3 * (size_t)(o + i) + d];
        for (int d = 0; d < 3; ++d) ctr[3 * c + d] /= n;
    }
    rc = ensure_staging(s, sizeof(double) * X.size());
    if (rc) return rc;
    HEMO_CU(cudaMemcpy(s->ctr, ctr.data(), sizeof(double) * ctr.size(), cudaMemcpyHostToDevice));
    HEMO_CU(cudaMemcpy(s->staging, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice));
    if (is_f64(s)) launch_set_vertices<double>(make_view<double>(s), (const double *)s->staging, s->stream);
    else launch_set_vertices<float>(make_view<float>(s), (const double *)s->staging, s->stream);
    HEMO_CU(cudaGetLastError());
    if ((rc = adapt_restart(s))) return rc;
    return hemo_sync(s);
}

int hemo_get_bins(hemo_sim *s, int32_t *key, int32_t *perm, int32_t *start) {
    NvtxRange nvtx_("hemo_get_bins");
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (s->nv) {
        if (is_f64(s)) launch_bins<double>(make_view<double>(s), s->stream, true);
        else launch_bins<float>(make_view<float>(s), s->stream, true);
        HEMO_CU(cudaGetLastError());
    }
    if ((rc = copy_out(s, key, s->key, sizeof(int) * s->nv))) return rc;
    if ((rc = copy_out(s, perm, s->perm, sizeof(int) * s->nv))) return rc;
    if ((rc = copy_out(s, start, s->start, sizeof(int) * (s->nbins + 1)))) return rc;
    return hemo_sync(s);
}

int hemo_set_phase_timing(hemo_sim *s, int on) {
    if (!s) return fail(HEMO_ERR_ARG, "null simulation");
    if ((bool)on == s->timing) return HEMO_OK;
    HEMO_CU(cudaStreamSynchronize(s->stream));
    if (on && !s->tev[0])
        for (int k = 0; k <= HEMO_NUM_PHASES; ++k) HEMO_CU(cudaEventCreate(&s->tev[k]));
    for (int k = 0; k < hemo_sim::NGRAPH; ++k)
        if (s->graph[k]) {
            cudaGraphExecDestroy(s->graph[k]);
            s->graph[k] = nullptr;
        }
    s->last_graph = -1;
    s->timing = on != 0;
    return HEMO_OK;
}

int hemo_get_phase_times(hemo_sim *s, float *ms, int *kernels_per_step) {
    if (!s || !ms) return fail(HEMO_ERR_ARG, "null pointer");
    if (!s->timing || s->last_graph < 0) return fail(HEMO_ERR_STATE, "phase timing is off or no timed step ran");
    HEMO_CU(cudaStreamSynchronize(s->stream));
    for (int k = 0; k < HEMO_NUM_PHASES; ++k) HEMO_CU(cudaEventElapsedTime(ms + k, s->tev[k], s->tev[k + 1]));
    if (kernels_per_step) *kernels_per_step = s->graph_kernels[s->last_graph];
    return HEMO_OK;
}

void hemo_destroy(hemo_sim *s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    clear_segment_graphs(s);
    for (int k = 0; k <= HEMO_NUM_PHASES; ++k)
        if (s->tev[k]) cudaEventDestroy(s->tev[k]);
    for (int k = 0; k < hemo_sim::NGRAPH; ++k)
        if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
    if (s->ev) cudaEventDestroy(s->ev);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->status_host) cudaFreeHost(s->status_host);
    std::vector<void *> all = s->allocs;
    for (void *p : all) dfree(s, p);
    cudaGetLastError();
    delete s;
}

}  // extern "C"
