// Reverse mode (adjoint) of the lattice part of the coupled step, for the
// differentiation form: gradients of a loss of the final vertex positions
// with respect to the membrane moduli, the wall velocity and the body force.
//
// Forward step n on the lattice (Sec. 2.2, 2.3, 2.5), natural layout:
//   collision at a fluid node: rho = sum f, u = (sum f c + F/2) / rho,
//     f*_i = (1 - w) f_i + w f^eq_i(rho, u) + S_i(u, F)            (BGK + Guo)
//   streaming: f'_i(x) = f*_i(x - c_i), or at a wall x - c_i:
//     f'_i(x) = f*_opp(i)(x) - 6 w_i rho(x) (c_opp(i) . u_wall)   (bounce-back)
//   velocity: u'(x) = (sum f' c + F/2) / rho'(x); u' = u_wall at wall nodes.
// The adjoint runs these backwards: the moments transpose adds
// lambda_u (c - u') / rho' to lambda_f' and lambda_u / (2 rho') to lambda_F;
// the forward step records rho and the collision velocity at each fluid node
// so that the collision transpose needs no populations;
// the streaming transpose pulls lambda_f* from the node each population
// streamed to (bounce-back: from the node itself); the collision transpose
// goes through (rho, u):
//   lambda_f_j = (1 - w) lambda*_j + g_rho + (c_j - u) . g_u / rho + lambda_rho,
//   g_rho = w sum_i lambda*_i f^eq_i / rho,
//   g_u = sum_i lambda*_i (w df^eq_i/du + dS_i/du),
//   lambda_F += sum_i lambda*_i dS_i/dF + g_u / (2 rho).
// Gradients accumulate in FP64 (per block in two-float precision first):
// wall-velocity scale s (u_wall = s u_given):
// sum over wall nodes of lambda_u . u_wall plus the bounce-back terms;
// body force g: sum over fluid nodes of lambda_F.
#include <type_traits>

#include "hemo_internal.cuh"

namespace hemo {

namespace {

inline int nblocks(long long n, int b) { return (int)((n + b - 1) / b); }

// block-wide sum of K per-thread values into the FP64 accumulators out (one
// atomic per block and value); warps reduce in two-float precision (Acc),
// only the per-warp totals are combined in FP64
template <typename R, int K>
__device__ void block_add(const R (&val)[K], double *out) {
    __shared__ double part[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    Acc<R> a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        a[k].add(val[k]);
        for (int o = 16; o > 0; o >>= 1) a[k].add_shfl(o);
    }
    if (lane == 0)
        for (int k = 0; k < K; ++k) part[k][wid] = a[k].value();
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0;
        for (int w = 0; w < nw; ++w) t += part[threadIdx.x][w];
        if (t != 0.0) atomicAdd(out + threadIdx.x, t);
    }
}

// transpose of u' = (sum f' c + F/2) / rho' (fluid) and u' = u_wall (walls).
// The contribution to the adjoint of f'_i at a fluid node is
// (c_i . lamu - lamu . u') / rho'; it is kept per node as four numbers and
// added by the streaming transpose when it pulls the population.
template <typename R>
__global__ void __launch_bounds__(256) adj_moments_kernel(View<R> v, AdjView<R> a) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    R ds[1] = {R(0)};
    if (n < v.N) {
        const size_t N = (size_t)v.N;
        const R lu[3] = {a.lamu[n], a.lamu[N + n], a.lamu[2 * N + n]};
        const int id = v.ntype[n] & 0x7f;
        if (id) {
            if (id >= 2) ds[0] = lu[0] * v.uw[id][0] + lu[1] * v.uw[id][1] + lu[2] * v.uw[id][2];
            for (int k = 0; k < 3; ++k) a.lamF[k * N + n] = R(0);
            for (int k = 0; k < 4; ++k) a.amom[k * N + n] = R(0);
        } else {
            const R ir = R(1) / a.rho1[n];
            const R lu_u = lu[0] * a.up[n] + lu[1] * a.up[N + n] + lu[2] * a.up[2 * N + n];
            for (int k = 0; k < 3; ++k) {
                a.amom[k * N + n] = lu[k] * ir;
                a.lamF[k * N + n] = R(0.5) * lu[k] * ir;
            }
            a.amom[3 * N + n] = -lu_u * ir;
        }
    }
    block_add<R, 1>(ds, a.grad + 4 * a.ntypes);
}

// transpose of streaming (pull, with the moments term of the pulled
// population) and of the collision at fluid node n
template <typename R>
__global__ void __launch_bounds__(256) adj_collide_kernel(View<R> v, AdjView<R> a) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    R acc[4] = {R(0), R(0), R(0), R(0)};  // wall-velocity scale, g_x, g_y, g_z
    if (n < v.N && !(v.ntype[n] & 0x7f)) {
        const size_t N = (size_t)v.N;
        const uint8_t nt = v.ntype[n];
        const uint64_t lk = (nt & 0x80) ? v.links[n] : 0ull;
        const Nbr o = make_nbr(v, n);
        // forward collision quantities, as the collision computed them
        const R rho = a.rec[n];
        const R u[3] = {a.rec[N + n], a.rec[2 * N + n], a.rec[3 * N + n]};
        const R F[3] = {v.F[n], v.F[N + n], v.F[2 * N + n]};
        const R ir = R(1) / rho;
        const R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const R om = v.omega, s0 = R(1) - R(0.5) * om;
        // pulled adjoint of the post-collision populations
        R ls[Q];
        R lrho = R(0);
        R dsw = R(0);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int code = link_code(lk, j);
            if (code) {  // bounced back into opp(j) at n
                const R lj = a.lamf_in[(size_t)opp(j) * N + n] -
                             (R(cx(j)) * a.amom[n] + R(cy(j)) * a.amom[N + n] + R(cz(j)) * a.amom[2 * N + n]) +
                             a.amom[3 * N + n];
                ls[j] = lj;
                const R cw = R(cx(j)) * v.uw[code][0] + R(cy(j)) * v.uw[code][1] + R(cz(j)) * v.uw[code][2];
                lrho -= R(6) * R(wgt(j)) * cw * lj;
                dsw -= R(6) * R(wgt(j)) * rho * cw * lj;
            } else {
                const size_t m = n + o.of(cx(j), cy(j), cz(j));
                R lj = a.lamf_in[(size_t)j * N + m] + a.amom[3 * N + m];
                if (cx(j)) lj += cx(j) > 0 ? a.amom[m] : -a.amom[m];
                if (cy(j)) lj += cy(j) > 0 ? a.amom[N + m] : -a.amom[N + m];
                if (cz(j)) lj += cz(j) > 0 ? a.amom[2 * N + m] : -a.amom[2 * N + m];
                ls[j] = lj;
            }
        }
        R grho = R(0), gu[3] = {R(0), R(0), R(0)}, lF[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R w = R(wgt(i));
            const R ci[3] = {R(cx(i)), R(cy(i)), R(cz(i))};
            const R cu = ci[0] * u[0] + ci[1] * u[1] + ci[2] * u[2];
            const R cF = ci[0] * F[0] + ci[1] * F[1] + ci[2] * F[2];
            const R feq = w * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
            grho += ls[i] * feq;
            for (int k = 0; k < 3; ++k) {
                const R dfeq = w * rho * (R(3) * ci[k] + R(9) * cu * ci[k] - R(3) * u[k]);
                const R dS = s0 * w * (R(-3) * F[k] + R(9) * cF * ci[k]);
                gu[k] += ls[i] * (om * dfeq + dS);
                lF[k] += ls[i] * s0 * w * (R(3) * (ci[k] - u[k]) + R(9) * cu * ci[k]);
            }
        }
        grho *= om * ir;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const R cgu = (R(cx(j)) - u[0]) * gu[0] + (R(cy(j)) - u[1]) * gu[1] + (R(cz(j)) - u[2]) * gu[2];
            a.lamf_out[(size_t)j * N + n] = (R(1) - om) * ls[j] + grho + cgu * ir + lrho;
        }
        for (int k = 0; k < 3; ++k) {
            const R tot = a.lamF[k * N + n] + lF[k] + R(0.5) * gu[k] * ir;
            a.lamF[k * N + n] = tot;
            acc[1 + k] = tot;
        }
        acc[0] = dsw;
    } else if (n < v.N) {
        const size_t N = (size_t)v.N;
        for (int j = 0; j < Q; ++j) a.lamf_out[(size_t)j * N + n] = R(0);
    }
    block_add<R, 4>(acc, a.grad + 4 * a.ntypes);
}

}  // namespace

template <typename R>
void launch_adj_moments(const View<R> &v, const AdjView<R> &a, cudaStream_t st) {
    adj_moments_kernel<R><<<nblocks(v.N, 256), 256, 0, st>>>(v, a);
}

template <typename R>
void launch_adj_collide(const View<R> &v, const AdjView<R> &a, cudaStream_t st) {
    adj_collide_kernel<R><<<nblocks(v.N, 256), 256, 0, st>>>(v, a);
}

#define HEMO_INST(R)                                                                  \
    template void launch_adj_moments<R>(const View<R> &, const AdjView<R> &, cudaStream_t); \
    template void launch_adj_collide<R>(const View<R> &, const AdjView<R> &, cudaStream_t);
HEMO_INST(double)
HEMO_INST(float)

}  // namespace hemo
