// Explicit fourth-order Runge-Kutta for scalar fields in a self-consistently
// expanding background (paper section 4.3.1), FP64: the non-symplectic
// reference integrator of the paper, kept for comparisons with the
// velocity-Verlet family.
//
// The scheme integrates (phi, v = phi', a, b) with
//   phi' = v,  v' = k = a^{-2(1-alpha)} L[phi] - (3-alpha)(b/a) v - a^{2 alpha} dV/dphi,
//   a' = b,    b' = K_a[a, E_K, E_G, E_V],  E_K = sum <v^2>/(2 a^{2 alpha}),
// stages y^(p) = y(n0) + dt b_{p,p-1} d^(p-1) (b_21 = b_32 = 1/2, b_43 = 1) and
// y(n0+1) = y(n0) + dt (d^(1) + 2 d^(2) + 2 d^(3) + d^(4))/6.
//
// Storage: full fields (no mean/fluctuation split) in four copies -- the
// state Y, two ping-pong stage copies and the accumulator A.  One pass per
// stage reads the stage state (7-point stencil through L1/L2), forms its
// derivatives, adds them into A and writes the next stage state Y + c dt d in
// the same sweep; the fourth pass writes Y = A + dt d/6.  The volume sums of
// the stage feed K_a in the last block, which advances a and b through the
// same stages.  At the boundaries of an evolve call the Hamiltonian momenta
// a^{3-alpha} phi' of the rest of the library are converted to v and back.
#include <math.h>

#include "cl_internal.cuh"
#include "scalar_common.cuh"

namespace cl {

struct Rk4Args {
    const double* T[4];  // stage state: phi_f (f < nf), v_f (nf + f)
    const double* Y[4];  // state at n0 (stages 2, 3: pointwise)
    double* A[4];        // accumulator (read-modify-write; written from Y at stage 1)
    double* out[4];      // next stage state, or the new Y at stage 4
    DevState* st;
    double* partials;
    unsigned int* counter;
    ModelConst mc;
    int stage;  // 0..3
    double dt;
};

// final weight of stage p (1/6, 1/3, 1/3, 1/6) and b_{p+1,p} (1/2, 1/2, 1) of the next stage
__host__ __device__ inline double rk_weight(int p) { return (p == 0 || p == 3) ? 1.0 / 6.0 : 1.0 / 3.0; }
__host__ __device__ inline double rk_next_c(int p) { return p == 2 ? 1.0 : 0.5; }

template <int NF, int P>
__global__ void __launch_bounds__(256) rk4_pass_kernel(const Rk4Args R) {
    DevState* st = R.st;
    if (st->error) return;
    constexpr int NS = 2 * NF + 2;  // sum v_f^2, sum (D+ phi_f)^2, V_p, V_q
    const int N = R.mc.N, p = R.stage;
    const double a = st->a, b = st->b, al = R.mc.alpha;
    const double c1 = pow(a, -2.0 * (1.0 - al)), c2 = (3.0 - al) * b / a, c3 = pow(a, 2.0 * al);
    const double idx2 = R.mc.idx2, lam = R.mc.lam, q = R.mc.q;
    const double wdt = rk_weight(p) * R.dt, cdt = p < 3 ? rk_next_c(p) * R.dt : 0.0;
    const size_t n3 = (size_t)N * N * N;
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
        const size_t xp = i - x + (x + 1 == N ? 0 : x + 1), xm = i - x + (x == 0 ? N - 1 : x - 1);
        const size_t NN = (size_t)N * N;
        const size_t yp = i + (size_t)((y + 1 == N ? 0 : y + 1) - y) * N, ym = i + (size_t)((y == 0 ? N - 1 : y - 1) - y) * N;
        const size_t zp = i + (size_t)((z + 1 == N ? 0 : z + 1) - z) * NN, zm = i + (size_t)((z == 0 ? N - 1 : z - 1) - z) * NN;
        double ph[NF], lap[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const double* F = R.T[f];
            const double c = __ldg(F + i), fxp = __ldg(F + xp), fyp = __ldg(F + yp), fzp = __ldg(F + zp);
            ph[f] = c;
            lap[f] = (fxp + __ldg(F + xm) + fyp + __ldg(F + ym) + fzp + __ldg(F + zm) - 6.0 * c) * idx2;
            acc[NF + f] += (fxp - c) * (fxp - c) + (fyp - c) * (fyp - c) + (fzp - c) * (fzp - c);
        }
        // full-field potential force: the split polynomials with a zero mean
        double F[2];
        F[0] = lam * Power<double, P>::dforce(0.0, ph[0]);
        acc[2 * NF] += lam * Power<double, P>::dvalue(0.0, ph[0]);
        F[1] = 0.0;
        if (NF > 1) {
            const double d0 = ph[0], d1 = ph[NF > 1 ? 1 : 0];
            F[0] += q * d1 * d1 * d0;
            F[1] = q * d0 * d0 * d1;
            acc[2 * NF + 1] += 0.5 * q * d0 * d0 * d1 * d1;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const double v = __ldg(R.T[NF + f] + i);
            const double k = c1 * lap[f] - c2 * v - c3 * F[f];
            acc[f] += v * v;
            // derivatives of (phi, v) at this stage: (v, k)
            const double yphi = p == 0 ? ph[f] : (p < 3 ? __ldg(R.Y[f] + i) : 0.0);
            const double yv = p == 0 ? v : (p < 3 ? __ldg(R.Y[NF + f] + i) : 0.0);
            if (p == 0) {
                R.A[f][i] = yphi + wdt * v;
                R.A[NF + f][i] = yv + wdt * k;
            } else if (p < 3) {
                R.A[f][i] += wdt * v;
                R.A[NF + f][i] += wdt * k;
            }
            if (p < 3) {
                R.out[f][i] = yphi + cdt * v;
                R.out[NF + f][i] = yv + cdt * k;
            } else {
                R.out[f][i] = R.A[f][i] + wdt * v;
                R.out[NF + f][i] = R.A[NF + f][i] + wdt * k;
            }
        }
    }
    // block reduction, partials, last block
    __shared__ double red[8][NS];
    const int lin = threadIdx.x, lane = lin & 31, warp = lin >> 5, nwarps = (blockDim.x + 31) >> 5;
    const int nlanes = min(32, (int)blockDim.x - 32 * warp);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const double v = partial_warp_sum(acc[s], lane, nlanes);
        if (lane == 0) red[warp][s] = v;
    }
    __syncthreads();
    if (lin < NS) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += red[w][lin];
        R.partials[(size_t)blockIdx.x * NS + lin] = t;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int last;
    if (lin == 0) last = (atomicAdd(R.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[NS];
    const double invV = 1.0 / (double)n3;
    for (int s = warp; s < NS; s += nwarps) {
        double ks = 0.0, kc = 0.0;
        for (int bl = lane; bl < (int)gridDim.x; bl += nlanes) {
            const double yk = __ldcg(&R.partials[(size_t)bl * NS + s]) - kc, tk = ks + yk;
            kc = (tk - ks) - yk;
            ks = tk;
        }
        const double r = partial_warp_sum(ks - kc, lane, nlanes);
        if (lane == 0) tot[s] = r * invV;
    }
    __syncthreads();
    if (lin != 0) return;
    *R.counter = 0u;
    const ModelConst& mc = R.mc;
    double EK[2] = {0, 0}, EG[2] = {0, 0};
    for (int f = 0; f < NF; ++f) {
        EK[f] = tot[f] / (2.0 * pow(a, 2.0 * al));
        EG[f] = tot[NF + f] * idx2 / (2.0 * a * a);
    }
    const double EV1 = tot[2 * NF], EV2 = NF > 1 ? tot[2 * NF + 1] : 0.0;
    const double EKt = EK[0] + EK[1], EGt = EG[0] + EG[1], EVt = EV1 + EV2;
    if (!isfinite(EKt + EGt + EVt)) {
        st->error = CL_ERR_NONFINITE;
        return;
    }
    const double ka = Ka_of(mc, a, EKt, EGt, EVt);
    if (p == 0) {  // stage 1 is the state at n0
        st->rk[0] = a;
        st->rk[1] = b;
        st->E[0] = EK[0]; st->E[1] = EK[1]; st->E[2] = EG[0]; st->E[3] = EG[1]; st->E[4] = EV1; st->E[5] = EV2;
        const double rhs = hubble_rhs(mc, a, EKt + EGt + EVt);
        st->hc = rhs > 0 ? fabs(b * b - rhs) / rhs : 0.0;
        st->rk[2] = a + wdt * b;
        st->rk[3] = b + wdt * ka;
    } else {
        st->rk[2] += wdt * b;
        st->rk[3] += wdt * ka;
    }
    if (p < 3) {  // next stage: a^(p+1) = a0 + c dt b^(p), b^(p+1) = b0 + c dt k_a^(p)
        st->a = st->rk[0] + cdt * b;
        st->b = st->rk[1] + cdt * ka;
    } else {
        st->a = st->rk[2];
        st->b = st->rk[3];
        st->t += R.dt;
        set_kick_powers(st, mc, st->a);
    }
}

// Enter: full fields and velocities v = pi / a^{3-alpha} from the stored
// mean + (array - pending shift) representation; the means become zero.
__global__ void rk4_enter_kernel(double* phi0, double* phi1, double* pi0, double* pi1, int nf, size_t n,
                                 const DevState* st, double alpha) {
    const double ia = pow(st->a, -(3.0 - alpha));
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        phi0[i] = st->phibar[0] + (phi0[i] - st->sphi[0]);
        pi0[i] = (st->pibar[0] + (pi0[i] - st->spi[0])) * ia;
        if (nf > 1) {
            phi1[i] = st->phibar[1] + (phi1[i] - st->sphi[1]);
            pi1[i] = (st->pibar[1] + (pi1[i] - st->spi[1])) * ia;
        }
    }
}

__global__ void rk4_zero_means_kernel(DevState* st) {
    for (int f = 0; f < kMaxComp; ++f) {
        st->phibar[f] = 0.0;
        st->pibar[f] = 0.0;
        st->sphi[f] = 0.0;
        st->spi[f] = 0.0;
    }
    st->cd = 0.0;
}

// Leave: Hamiltonian momenta pi = a^{3-alpha} v.
__global__ void rk4_leave_kernel(double* pi0, double* pi1, int nf, size_t n, const DevState* st, double alpha) {
    const double sa = pow(st->a, 3.0 - alpha);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        pi0[i] *= sa;
        if (nf > 1) pi1[i] *= sa;
    }
}

template <int NF, int P> static const void* rk4_kernel_p() { return (const void*)rk4_pass_kernel<NF, P>; }

static cudaError_t rk4_launch(Lattice* L, const Rk4Args& R, cudaStream_t s) {
    const int grid = std::min(L->sm_count * 8, kMaxBlocks);
    const int nf = L->mc.nf, P = L->mc.pexp;
#define CL_RK4_CASE(NFV, PV) \
    if (nf == NFV && P == PV) { rk4_pass_kernel<NFV, PV><<<grid, 256, 0, s>>>(R); return cudaGetLastError(); }
    CL_RK4_CASE(1, 2) CL_RK4_CASE(1, 4) CL_RK4_CASE(1, 6) CL_RK4_CASE(2, 2) CL_RK4_CASE(2, 4) CL_RK4_CASE(2, 6)
#undef CL_RK4_CASE
    return cudaErrorInvalidValue;
}

// m RK4 steps on copy `cur` (the state stays in that copy).
cudaError_t rk4_enqueue(Lattice* L, long long m, int cur, cudaStream_t s) {
    const int nf = L->mc.nf;
    const size_t n = (size_t)L->mc.N * L->mc.N * L->mc.N;
    double* Y[4] = {nullptr, nullptr, nullptr, nullptr};
    double* T0[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int a = 0; a < 2 * nf; ++a) {
        Y[a] = static_cast<double*>(L->buf.f[cur][a]);
        T0[a] = static_cast<double*>(L->buf.f[1 - cur][a]);
    }
    const int eg = L->sm_count * 4;
    rk4_enter_kernel<<<eg, 256, 0, s>>>(Y[0], nf > 1 ? Y[1] : nullptr, Y[nf], nf > 1 ? Y[nf + 1] : nullptr, nf, n,
                                        L->buf.st, L->mc.alpha);
    rk4_zero_means_kernel<<<1, 1, 0, s>>>(L->buf.st);
    cudaError_t e = cudaGetLastError();
    for (long long j = 0; j < m && e == cudaSuccess; ++j) {
        for (int p = 0; p < 4 && e == cudaSuccess; ++p) {
            Rk4Args R;
            // stage inputs: Y, T0, T1, T0; outputs: T0, T1, T0, Y
            double* const* in = p == 0 ? Y : (p == 2 ? (double* const*)L->rk_T1 : T0);
            double* const* out = p == 0 ? T0 : (p == 1 ? (double* const*)L->rk_T1 : (p == 2 ? T0 : Y));
            for (int a = 0; a < 4; ++a) {
                R.T[a] = a < 2 * nf ? in[a] : nullptr;
                R.Y[a] = a < 2 * nf ? Y[a] : nullptr;
                R.A[a] = a < 2 * nf ? static_cast<double*>(L->rk_A[a]) : nullptr;
                R.out[a] = a < 2 * nf ? out[a] : nullptr;
            }
            R.st = L->buf.st;
            R.partials = L->buf.partials;
            R.counter = L->buf.counter;
            R.mc = L->mc;
            R.stage = p;
            R.dt = L->grid.dt;
            e = rk4_launch(L, R, s);
        }
    }
    if (e == cudaSuccess) {
        rk4_leave_kernel<<<eg, 256, 0, s>>>(Y[nf], nf > 1 ? Y[nf + 1] : nullptr, nf, n, L->buf.st, L->mc.alpha);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace cl
