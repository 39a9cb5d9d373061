// Gauss-Legendre implicit Runge-Kutta for scalar fields in a self-consistently
// expanding background (paper sections 3.4.2 and 4.3.3, Scheme II: the
// Hamiltonian variables of the rest of the library), FP64.
//
//   y = (phi, pi, a, b),  F(y) = (a^{-(3-alpha)} pi, a^{1+alpha} L[phi] - a^{3+alpha} V'(phi), b, K_a[a, E(y)]),
//   Y^(l) = y(n0) + dt sum_m A_lm D^(m),   D^(l) = F(Y^(l)),   l = 1..s,
//   y(n0 + 1) = y(n0) + dt sum_m c_m D^(m),
// with the s-stage Gauss-Legendre tableau (order 2s), computed here from its
// definition: collocation at the roots tau_i of P_s(2 tau - 1), A_ij the integral
// of the j-th Lagrange polynomial from 0 to tau_i, c_j its integral over [0, 1].
//
// The stage equations are solved by Jacobi fixed-point sweeps from D = 0 (the
// first sweep gives F(y(n0)) for every stage).  One kernel per sweep forms
// every stage state on the fly (the stencil of phi^(l) included), writes the
// new stage derivatives into the other of two buffers and reduces the stage
// energies and the change of D; its last block updates the scalar stages and
// raises a device-side flag once ||D_new - D_old|| <= tol ||D_new||, after which
// the remaining sweeps of the step return at once (the schedule of launches is
// fixed, so an evolve call is still one CUDA graph).  The arrays hold full
// fields in FP64 (the means are folded in when an evolve call starts).
#include <math.h>

#include <vector>

#include "cl_internal.cuh"
#include "scalar_common.cuh"

namespace cl {

constexpr int kGlMaxS = 5;

struct GlArgs {
    const double* Y[4];              // state at n0: phi_f (f < nf), pi_f (nf + f)
    double* D[2][kGlMaxS][4];        // stage derivatives, two buffers: dphi_f, dpi_f
    double A[kGlMaxS][kGlMaxS], c[kGlMaxS];
    int s;
    double dt, tol;
    DevState* st;
    double* partials;
    unsigned int* counter;
    ModelConst mc;
};

template <int NF, int P>
__global__ void __launch_bounds__(256) gl_sweep_kernel(const GlArgs G) {
    DevState* st = G.st;
    if (st->error || st->gl_conv) return;
    constexpr int NSS = 3;                          // per stage: sum pi^2, sum (D+ phi)^2, sum V
    constexpr int NS = NSS * kGlMaxS + 2;           // + |D_new - D_old|^2, |D_new|^2
    const int s = G.s, N = G.mc.N;
    const int bo = st->gl_cur, bn = 1 - bo;
    const double dt = G.dt, al = G.mc.alpha, idx2 = G.mc.idx2, lam = G.mc.lam, q = G.mc.q;
    double a_l[kGlMaxS];
    for (int l = 0; l < s; ++l) {
        double x = st->rk[0];
        for (int m = 0; m < s; ++m) x += dt * G.A[l][m] * st->gl_Da[bo][m];
        a_l[l] = x;
    }
    const size_t n3 = (size_t)N * N * N;
    double acc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[k] = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
        const size_t NN = (size_t)N * N;
        const size_t nbr[6] = {i - x + (x + 1 == N ? 0 : x + 1), i - x + (x == 0 ? N - 1 : x - 1),
                               i + (size_t)((y + 1 == N ? 0 : y + 1) - y) * N, i + (size_t)((y == 0 ? N - 1 : y - 1) - y) * N,
                               i + (size_t)((z + 1 == N ? 0 : z + 1) - z) * NN, i + (size_t)((z == 0 ? N - 1 : z - 1) - z) * NN};
        for (int l = 0; l < s; ++l) {
            // stage state: Y + dt sum_m A_lm D^(m) at the site and its six neighbours
            double ph[NF], lap[NF], pi_l[NF];
            for (int f = 0; f < NF; ++f) {
                auto stage_phi = [&](size_t k) {
                    double v = __ldg(G.Y[f] + k);
                    for (int m = 0; m < s; ++m) v += dt * G.A[l][m] * G.D[bo][m][f][k];
                    return v;
                };
                const double c0 = stage_phi(i);
                double sum = 0.0, g2 = 0.0;
                for (int j = 0; j < 6; ++j) {
                    const double v = stage_phi(nbr[j]);
                    sum += v;
                    if ((j & 1) == 0) g2 += (v - c0) * (v - c0);  // forward neighbours
                }
                ph[f] = c0;
                lap[f] = (sum - 6.0 * c0) * idx2;
                acc[NSS * l + 1] += g2;
                double pv = __ldg(G.Y[NF + f] + i);
                for (int m = 0; m < s; ++m) pv += dt * G.A[l][m] * G.D[bo][m][NF + f][i];
                pi_l[f] = pv;
            }
            double F[2];
            F[0] = lam * Power<double, P>::dforce(0.0, ph[0]);
            acc[NSS * l + 2] += lam * Power<double, P>::dvalue(0.0, ph[0]);
            F[1] = 0.0;
            if (NF > 1) {
                const double d0 = ph[0], d1 = ph[NF > 1 ? 1 : 0];
                F[0] += q * d1 * d1 * d0;
                F[1] = q * d0 * d0 * d1;
                acc[NSS * l + 2] += 0.5 * q * d0 * d0 * d1 * d1;
            }
            const double A1 = pow(a_l[l], 1.0 + al), A3 = pow(a_l[l], 3.0 + al), cd = pow(a_l[l], -(3.0 - al));
            for (int f = 0; f < NF; ++f) {
                const double dphi = cd * pi_l[f], dpi = A1 * lap[f] - A3 * F[f];
                const double o1 = G.D[bo][l][f][i], o2 = G.D[bo][l][NF + f][i];
                G.D[bn][l][f][i] = dphi;
                G.D[bn][l][NF + f][i] = dpi;
                acc[NSS * l] += pi_l[f] * pi_l[f];
                acc[NS - 2] += (dphi - o1) * (dphi - o1) + (dpi - o2) * (dpi - o2);
                acc[NS - 1] += dphi * dphi + dpi * dpi;
            }
        }
    }
    // block reduction, partials, last block
    __shared__ double red[8][NS];
    const int lin = threadIdx.x, lane = lin & 31, warp = lin >> 5, nwarps = (blockDim.x + 31) >> 5;
    const int nlanes = min(32, (int)blockDim.x - 32 * warp);
    for (int k = 0; k < NS; ++k) {
        const double v = partial_warp_sum(acc[k], lane, nlanes);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (lin < NS) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += red[w][lin];
        G.partials[(size_t)blockIdx.x * NS + lin] = t;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int last;
    if (lin == 0) last = (atomicAdd(G.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[NS];
    for (int k = warp; k < NS; k += nwarps) {
        double ks = 0.0, kc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += nlanes) {
            const double yk = __ldcg(&G.partials[(size_t)b * NS + k]) - kc, tk = ks + yk;
            kc = (tk - ks) - yk;
            ks = tk;
        }
        const double r = partial_warp_sum(ks - kc, lane, nlanes);
        if (lane == 0) tot[k] = r;  // raw sums (volume averages taken below)
    }
    __syncthreads();
    if (lin != 0) return;
    *G.counter = 0u;
    const double invV = 1.0 / (double)n3;
    double dd = tot[NS - 2], nn = tot[NS - 1];
    for (int l = 0; l < s; ++l) {
        double bl = st->rk[1];
        for (int m = 0; m < s; ++m) bl += dt * G.A[l][m] * st->gl_Db[bo][m];
        const double a = a_l[l];
        const double EK = tot[NSS * l] * invV / (2.0 * pow(a, 6.0));
        const double EG = tot[NSS * l + 1] * invV * idx2 / (2.0 * a * a);
        const double EV = tot[NSS * l + 2] * invV;
        if (!isfinite(EK + EG + EV)) {
            st->error = CL_ERR_NONFINITE;
            return;
        }
        const double da = bl, db = Ka_of(G.mc, a, EK, EG, EV);
        dd += (da - st->gl_Da[bo][l]) * (da - st->gl_Da[bo][l]) + (db - st->gl_Db[bo][l]) * (db - st->gl_Db[bo][l]);
        nn += da * da + db * db;
        st->gl_Da[bn][l] = da;
        st->gl_Db[bn][l] = db;
    }
    st->gl_cur = bn;
    st->gl_it += 1;
    if (dd <= G.tol * G.tol * nn) st->gl_conv = 1;
}

// y(n0 + 1) = y(n0) + dt sum_m c_m D^(m) from the latest buffer (pointwise);
// a step whose stage sweeps did not converge is not applied
__global__ void gl_final_kernel(const GlArgs G, int nf) {
    const DevState* st = G.st;
    if (st->error || !st->gl_conv) return;
    const int b = st->gl_cur;
    const size_t n3 = (size_t)G.mc.N * G.mc.N * G.mc.N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 2 * nf; ++k) {
            double v = G.Y[k][i];
            for (int m = 0; m < G.s; ++m) v += G.dt * G.c[m] * G.D[b][m][k][i];
            const_cast<double*>(G.Y[k])[i] = v;
        }
}

// start of a step: a0, b0 <- a, b; D = 0 (the arrays are cleared separately)
__global__ void gl_begin_kernel(DevState* st) {
    st->rk[0] = st->a;
    st->rk[1] = st->b;
    for (int m = 0; m < kGlMaxS; ++m) st->gl_Da[0][m] = st->gl_Db[0][m] = st->gl_Da[1][m] = st->gl_Db[1][m] = 0.0;
    st->gl_cur = 0;
    st->gl_conv = 0;
    st->gl_it = 0;
}

// end of a step: the scalars with the final weights.  Without convergence of
// the stage equations the step is refused: the error flag stops the lattice at
// the last completed step and the host reports CL_ERR_TIMEOUT.
__global__ void gl_end_kernel(DevState* st, ModelConst mc, int s, double dt, double c0, double c1, double c2,
                              double c3, double c4) {
    if (st->error) return;
    if (!st->gl_conv) {
        st->error = CL_ERR_TIMEOUT;
        return;
    }
    const double c[kGlMaxS] = {c0, c1, c2, c3, c4};
    const int b = st->gl_cur;
    double a = st->rk[0], bb = st->rk[1];
    for (int m = 0; m < s; ++m) {
        a += dt * c[m] * st->gl_Da[b][m];
        bb += dt * c[m] * st->gl_Db[b][m];
    }
    st->a = a;
    st->b = bb;
    st->t += dt;
    set_kick_powers(st, mc, a);
}

// fold the means into the arrays (full fields), zero the means and shifts
__global__ void gl_enter_kernel(double* phi0, double* phi1, double* pi0, double* pi1, int nf, size_t n,
                                const DevState* st) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        phi0[i] = st->phibar[0] + (phi0[i] - st->sphi[0]);
        pi0[i] = st->pibar[0] + (pi0[i] - st->spi[0]);
        if (nf > 1) {
            phi1[i] = st->phibar[1] + (phi1[i] - st->sphi[1]);
            pi1[i] = st->pibar[1] + (pi1[i] - st->spi[1]);
        }
    }
}

__global__ void gl_zero_means_kernel(DevState* st) {
    for (int f = 0; f < kMaxComp; ++f) st->phibar[f] = st->pibar[f] = st->sphi[f] = st->spi[f] = 0.0;
    st->cd = 0.0;
}

// Gauss-Legendre tableau from its definition: Newton on P_s for the nodes,
// exact integration of the Lagrange polynomials (coefficient arrays).
void gl_tableau(int s, double A[kGlMaxS][kGlMaxS], double c[kGlMaxS]) {
    std::vector<double> x(s);
    for (int i = 0; i < s; ++i) {
        double t = cos(M_PI * (i + 0.75) / (s + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;  // P_0, P_1; recurrence (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}
            for (int k = 1; k < s; ++k) {
                const double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            const double dp = s * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = t;
    }
    std::vector<double> tau(s);
    for (int i = 0; i < s; ++i) tau[i] = 0.5 * (1.0 - x[i]);  // increasing order
    for (int j = 0; j < s; ++j) {
        std::vector<double> poly(1, 1.0);  // coefficients of l_j, ascending powers
        for (int k = 0; k < s; ++k) {
            if (k == j) continue;
            std::vector<double> np(poly.size() + 1, 0.0);
            const double den = tau[j] - tau[k];
            for (size_t p = 0; p < poly.size(); ++p) {
                np[p + 1] += poly[p] / den;
                np[p] -= tau[k] * poly[p] / den;
            }
            poly.swap(np);
        }
        auto integral = [&](double u) {
            double v = 0.0, up = u;
            for (size_t p = 0; p < poly.size(); ++p, up *= u) v += poly[p] * up / (double)(p + 1);
            return v;
        };
        c[j] = integral(1.0);
        for (int i = 0; i < s; ++i) A[i][j] = integral(tau[i]);
    }
}

static cudaError_t gl_sweep_launch(Lattice* L, const GlArgs& G, cudaStream_t st) {
    const int grid = std::min(L->sm_count * 4, kMaxBlocks);
    const int nf = L->mc.nf, P = L->mc.pexp;
#define CL_GL_CASE(NFV, PV) \
    if (nf == NFV && P == PV) { gl_sweep_kernel<NFV, PV><<<grid, 256, 0, st>>>(G); return cudaGetLastError(); }
    CL_GL_CASE(1, 2) CL_GL_CASE(1, 4) CL_GL_CASE(1, 6) CL_GL_CASE(2, 2) CL_GL_CASE(2, 4) CL_GL_CASE(2, 6)
#undef CL_GL_CASE
    return cudaErrorInvalidValue;
}

// m Gauss-Legendre steps of the state in copy `cur`
cudaError_t gl_enqueue(Lattice* L, long long m, int cur, cudaStream_t s) {
    const int nf = L->mc.nf, stages = L->integ - CL_INT_GL2 + 2;
    const size_t n = (size_t)L->mc.N * L->mc.N * L->mc.N;
    GlArgs G;
    memset(&G, 0, sizeof(G));
    for (int k = 0; k < 2 * nf; ++k) G.Y[k] = static_cast<const double*>(L->buf.f[cur][k]);
    for (int b = 0; b < 2; ++b)
        for (int l = 0; l < stages; ++l)
            for (int k = 0; k < 2 * nf; ++k) G.D[b][l][k] = static_cast<double*>(L->gl_D[b][l][k]);
    gl_tableau(stages, G.A, G.c);
    G.s = stages;
    G.dt = L->grid.dt;
    G.tol = 1e-14;
    G.st = L->buf.st;
    G.partials = L->buf.partials;
    G.counter = L->buf.counter;
    G.mc = L->mc;
    double* Y[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 2 * nf; ++k) Y[k] = static_cast<double*>(L->buf.f[cur][k]);
    const int eg = L->sm_count * 4;
    gl_enter_kernel<<<eg, 256, 0, s>>>(Y[0], nf > 1 ? Y[1] : nullptr, Y[nf], nf > 1 ? Y[nf + 1] : nullptr, nf, n,
                                       L->buf.st);
    gl_zero_means_kernel<<<1, 1, 0, s>>>(L->buf.st);
    cudaError_t e = cudaGetLastError();
    const int maxit = 60;
    for (long long j = 0; j < m && e == cudaSuccess; ++j) {
        gl_begin_kernel<<<1, 1, 0, s>>>(L->buf.st);
        for (int l = 0; l < stages && e == cudaSuccess; ++l)
            for (int k = 0; k < 2 * nf && e == cudaSuccess; ++k) e = cudaMemsetAsync(G.D[0][l][k], 0, n * sizeof(double), s);
        for (int it = 0; it < maxit && e == cudaSuccess; ++it) e = gl_sweep_launch(L, G, s);
        if (e != cudaSuccess) break;
        gl_final_kernel<<<eg, 256, 0, s>>>(G, nf);
        gl_end_kernel<<<1, 1, 0, s>>>(L->buf.st, L->mc, stages, G.dt, G.c[0], G.c[1], G.c[2], G.c[3], G.c[4]);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace cl
