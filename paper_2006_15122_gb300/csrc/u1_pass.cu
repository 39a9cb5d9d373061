// Compact U(1) sector (paper section 5.3): a complex scalar phi with
// momentum pi = a^{3-alpha} phi' and link angles theta_i = e dx A_i
// (V_i = exp(-i theta_i)) with electric momenta piA_i = a^{1-alpha} F_0i.
//
// Kernels (section 5.3, both derived from one lattice action so that the
// discrete Gauss law holds exactly):
//   K_phi  = -a^{3+alpha} (lam/2)(|phi|^2 - v2) phi
//            + a^{1+alpha} sum_i (V_i phi(n+i) - 2 phi + V_i*(n-i) phi(n-i)) / dx^2
//   K_A,i  = a^{1+alpha} (2e/dx)(1/kappa) Im[phi*(n) V_i(n) phi(n+i)]
//            + a^{alpha-1}/(e dx^3) sum_{j!=i} [Im V_ij(n) - Im V_ij(n-j)],
//   V_ij(n) = V_i(n) V_j(n+i) V_i*(n+j) V_j*(n) = exp(-i theta_ij),
//   theta_ij(n) = theta_i(n) + theta_j(n+i) - theta_i(n+j) - theta_j(n),
// kappa = (w*/f*)^2.  Drifts (compact staggered leapfrog, section 5.3.1, and
// the compact velocity-Verlet VV2..VV10 of sections 5.3.2-5.3.3 with dt -> w_p dt):
//   phi <- phi + dt a_{1/2}^{-(3-alpha)} pi,
//   V_i <- exp(-i e dx dt a_{1/2}^{-(1-alpha)} piA_i) V_i  (theta_i += ..., wrapped to [-pi, pi)),
// the exact exponential of the link drift (unitary for any step).
// Non-compact formulation (section 5.2, mc.nc): the same kernels with sin theta_ij
// replaced by theta_ij (the lattice curl of curl A) and 1 - cos theta_ij by
// theta_ij^2/2 in E_G^A; the angles theta_i = e dx A_i are then not wrapped.
// Energies (section 5.4.1): E_K^phi = <|pi|^2>/a^6, E_G^phi = sum_i <|D_i^+ phi|^2>/a^2,
// E_V = <V>, E_K^A = kappa/(2a^4) sum_i <piA_i^2>,
// E_G^A = kappa/(a^4 e^2 dx^4) sum_{i<j} <1 - cos theta_ij>.
//
// One thread per site with a persistent grid-stride loop; neighbour values
// come through L1/L2 and are drifted on the fly, so each array is read once
// from HBM and written once per pass.  The last block does the FP64
// leapfrog/Friedmann update as in the scalar pass.
#include <math.h>

#include "cl_internal.cuh"
#include "gauge_finish.cuh"

namespace cl {

struct U1Args {
    const void* in[10];
    void* out[10];
    DevState* st;
    double* partials;
    unsigned int* counter;
    ModelConst mc;
    PassInfo pi;
    int write;
};



template <typename T> __device__ __forceinline__ T wrap_angle(T t) {
    const T twopi = T(6.283185307179586476925287);
    return t - twopi * rint(t / twopi);
}
template <typename T> __device__ __forceinline__ void sc(T x, T* s, T* c);
// FP32: the hardware approximation (the arguments are sums of at most four
// wrapped angles, |x| <= 4 pi); every thread evaluates a shared plaquette from
// the same inputs in the same order, so the cancellations behind the Gauss law
// stay exact
template <> __device__ __forceinline__ void sc<float>(float x, float* s, float* c) { __sincosf(x, s, c); }
template <> __device__ __forceinline__ void sc<double>(double x, double* s, double* c) { sincos(x, s, c); }
// link phases of the non-compact formulation: its angles are not wrapped, so FP32
// takes the range-reduced sincosf
template <typename T, bool NC> __device__ __forceinline__ void sc_link(T x, T* s, T* c) {
    if (sizeof(T) == 4 && NC) sincosf(float(x), reinterpret_cast<float*>(s), reinterpret_cast<float*>(c));
    else sc<T>(x, s, c);
}

// NC: the non-compact formulation (a separate instantiation, so the compact pass is unchanged)
template <typename T, bool NC>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) u1_pass_kernel(const U1Args A) {
    DevState* st = A.st;
    if (st->error) return;
    const int N = A.mc.N;
    const T cd = T(st->cd), cdA = T(st->cdA), A1 = T(st->A1), A3 = T(st->A3), Am = T(st->Am);
    const T h1 = T(A.pi.h1), h = T(A.pi.h);
    const T dx = T(A.mc.dx), idx = T(1.0 / A.mc.dx), idx2 = T(A.mc.idx2);
    const T lam = T(A.mc.lam), v2 = T(A.mc.vev2);
    const T cJ = T(2.0 * A.mc.e / A.mc.dx / A.mc.kappa), cB = T(1.0 / (A.mc.e * A.mc.dx * A.mc.dx * A.mc.dx));
    constexpr bool nc = NC;  // non-compact: the plaquette angle itself replaces sin, theta^2/2 replaces 1 - cos
    (void)dx;
    const T* PR = static_cast<const T*>(A.in[0]);
    const T* PIm = static_cast<const T*>(A.in[1]);
    const T* QR = static_cast<const T*>(A.in[2]);
    const T* QI = static_cast<const T*>(A.in[3]);
    const T* TH[3] = {static_cast<const T*>(A.in[4]), static_cast<const T*>(A.in[5]), static_cast<const T*>(A.in[6])};
    const T* EA[3] = {static_cast<const T*>(A.in[7]), static_cast<const T*>(A.in[8]), static_cast<const T*>(A.in[9])};
    const size_t n3 = (size_t)N * N * N;
    double acc[U1NS];
#pragma unroll
    for (int s = 0; s < U1NS; ++s) acc[s] = 0.0;
    T ts[U1NS];
#pragma unroll
    for (int s = 0; s < U1NS; ++s) ts[s] = T(0);
    int cnt = 0;

    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += stride) {
        // the grid's next chunk of sites into L2 while this one computes
        if (i + stride < n3) {
#pragma unroll
            for (int a = 0; a < 10; ++a) prefetch_l2(static_cast<const T*>(A.in[a]) + i + stride);
        }
        const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
        const int c[3] = {x, y, z};
        auto at = [&](int dxs, int dys, int dzs) -> size_t {
            int xx = x + dxs, yy = y + dys, zz = z + dzs;
            xx = xx < 0 ? xx + N : (xx >= N ? xx - N : xx);
            yy = yy < 0 ? yy + N : (yy >= N ? yy - N : yy);
            zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
            return ((size_t)zz * N + yy) * N + xx;
        };
        (void)c;
        // drifted values
        auto phr = [&](size_t k) { return __ldg(PR + k) + cd * __ldg(QR + k); };
        auto phi_ = [&](size_t k) { return __ldg(PIm + k) + cd * __ldg(QI + k); };
        auto th = [&](int d, size_t k) { return __ldg(TH[d] + k) + cdA * __ldg(EA[d] + k); };
        const T fr = phr(i), fi = phi_(i);
        const T pr = __ldg(QR + i), pim = __ldg(QI + i);
        T t0[3], ea[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) { t0[d] = th(d, i); ea[d] = __ldg(EA[d] + i); }
        // covariant Laplacian, current, gradient energy
        T lr = T(-6) * fr, li = T(-6) * fi, grad = T(0);
        T Kj[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int ox = d == 0, oy = d == 1, oz = d == 2;
            const size_t np = at(ox, oy, oz), nm = at(-ox, -oy, -oz);
            const T ur0 = phr(np), ui0 = phi_(np);
            T s, cc;
            sc_link<T, NC>(t0[d], &s, &cc);
            // V_i phi(n+i) = (cos t - i sin t)(ur0 + i ui0)
            const T ur = cc * ur0 + s * ui0, ui = cc * ui0 - s * ur0;
            const T tm = th(d, nm);
            T sm, cm;
            sc_link<T, NC>(tm, &sm, &cm);
            const T wr0 = phr(nm), wi0 = phi_(nm);
            // V_i*(n-i) phi(n-i) = (cos tm + i sin tm)(wr0 + i wi0)
            const T wr = cm * wr0 - sm * wi0, wi = cm * wi0 + sm * wr0;
            lr += ur + wr;
            li += ui + wi;
            const T gr = ur - fr, gi = ui - fi;
            grad += gr * gr + gi * gi;
            Kj[d] = cJ * (fr * ui - fi * ur);  // (2e/dx)(1/kappa) Im[phi* V_i phi(n+i)]
        }
        // plaquettes at n, one per unordered pair (theta_ji = -theta_ij): pairs (0,1), (0,2), (1,2)
        T sp[3], eB = T(0);
#pragma unroll
        for (int pr_ = 0; pr_ < 3; ++pr_) {
            const int ii = pr_ == 2 ? 1 : 0, jj = pr_ == 0 ? 1 : 2;
            const int oix = ii == 0, oiy = ii == 1, oiz = ii == 2;
            const int ojx = jj == 0, ojy = jj == 1, ojz = jj == 2;
            const T pn = t0[ii] + th(jj, at(oix, oiy, oiz)) - th(ii, at(ojx, ojy, ojz)) - t0[jj];
            if (nc) {
                sp[pr_] = pn;
                eB += T(0.5) * pn * pn;
            } else {
                T cn;
                sc<T>(pn, &sp[pr_], &cn);
                eB += T(1) - cn;
            }
        }
        // forces: sum_j [Im V_ij(n) - Im V_ij(n-j)], Im V_ij = -sin(theta_ij)
        T mag[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int ii = 0; ii < 3; ++ii) {
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                if (jj == ii) continue;
                const int oix = ii == 0, oiy = ii == 1, oiz = ii == 2;
                const int ojx = jj == 0, ojy = jj == 1, ojz = jj == 2;
                const int pr_ = ii + jj - 1;  // (0,1) -> 0, (0,2) -> 1, (1,2) -> 2
                const T sn = ii < jj ? sp[pr_] : -sp[pr_];
                const T pm = th(ii, at(-ojx, -ojy, -ojz)) + th(jj, at(oix - ojx, oiy - ojy, oiz - ojz)) - t0[ii] -
                             th(jj, at(-ojx, -ojy, -ojz));
                T smm = pm, cmm;
                if (!nc) sc<T>(pm, &smm, &cmm);
                mag[ii] += -sn + smm;
            }
        }
        const T mod2 = fr * fr + fi * fi;
        T dv;
        const T vpot = gauge_pot<T>(A.mc.gpot, A.mc.pexp, lam, v2, mod2, &dv);
        const T Kr = -A3 * dv * fr + A1 * lr * idx2, Ki = -A3 * dv * fi + A1 * li * idx2;
        const T prr = pr + h1 * Kr, pri = pim + h1 * Ki;
        const T por = pr + h * Kr, poi = pim + h * Ki;
        T sA = T(0), eo[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const T K = A1 * Kj[d] + Am * cB * mag[d];
            const T er = ea[d] + h1 * K;
            eo[d] = ea[d] + h * K;
            sA += er * er;
        }
        ts[0] += fr; ts[1] += fi; ts[2] += fr * fr; ts[3] += fi * fi;
        ts[4] += prr; ts[5] += pri; ts[6] += prr * prr + pri * pri;
        ts[7] += grad * idx2;
        ts[8] += vpot;
        ts[9] += sA;
        ts[10] += eB;
        if (A.write) {
            static_cast<T*>(A.out[0])[i] = fr;
            static_cast<T*>(A.out[1])[i] = fi;
            static_cast<T*>(A.out[2])[i] = por;
            static_cast<T*>(A.out[3])[i] = poi;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                static_cast<T*>(A.out[4 + d])[i] = nc ? t0[d] : wrap_angle(t0[d]);
                static_cast<T*>(A.out[7 + d])[i] = eo[d];
            }
        }
        if (++cnt == 64) {  // fold into FP64 every 64 sites
#pragma unroll
            for (int s = 0; s < U1NS; ++s) { acc[s] += double(ts[s]); ts[s] = T(0); }
            cnt = 0;
        }
    }
#pragma unroll
    for (int s = 0; s < U1NS; ++s) acc[s] += double(ts[s]);
    (void)idx;

    // block reduction, partials, last block
    __shared__ double red[8][U1NS];
    const int lin = threadIdx.x, lane = lin & 31, warp = lin >> 5, nwarps = (blockDim.x + 31) >> 5;
    const int nlanes = min(32, (int)blockDim.x - 32 * warp);
#pragma unroll
    for (int s = 0; s < U1NS; ++s) {
        const double v = partial_warp_sum(acc[s], lane, nlanes);
        if (lane == 0) red[warp][s] = v;
    }
    __syncthreads();
    if (lin < U1NS) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += red[w][lin];
        A.partials[(size_t)blockIdx.x * U1NS + lin] = t;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int last;
    if (lin == 0) last = (atomicAdd(A.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[U1NS];
    const double invV = 1.0 / (double)n3;
    for (int s = warp; s < U1NS; s += nwarps) {
        double ks = 0.0, kc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += nlanes) {
            const double xv = __ldcg(&A.partials[(size_t)b * U1NS + s]);
            const double yk = xv - kc, tk = ks + yk;
            kc = (tk - ks) - yk;
            ks = tk;
        }
        const double r = partial_warp_sum(ks - kc, lane, nlanes);
        if (lane == 0) tot[s] = r * invV;
    }
    __syncthreads();
    if (lin == 0) {
        *A.counter = 0u;
        u1_finish(st, tot, A.mc, A.pi);
    }
}

// Closing drift of the leapfrog (in place): phi += cd pi, theta += cdA piA (wrapped when compact).
template <typename T>
__global__ void u1_drift_kernel(T* pr, T* pim, const T* qr, const T* qi, T* t0, T* t1, T* t2, const T* e0,
                                const T* e1, const T* e2, size_t n, DevState* st, int nc) {
    if (st->error) return;
    const T cd = T(st->cd), cdA = T(st->cdA);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        pr[i] += cd * qr[i];
        pim[i] += cd * qi[i];
        const T a0 = t0[i] + cdA * e0[i], a1 = t1[i] + cdA * e1[i], a2 = t2[i] + cdA * e2[i];
        t0[i] = nc ? a0 : wrap_angle(a0);
        t1[i] = nc ? a1 : wrap_angle(a1);
        t2[i] = nc ? a2 : wrap_angle(a2);
    }
}

// Gauss-law residual G = sum_i D_i^- piA_i - (2e/kappa) Im[phi* pi] (section 5.2), FP64 sums.
template <typename T>
__global__ void u1_gauss_kernel(const T* pr, const T* pim, const T* qr, const T* qi, const T* e0, const T* e1,
                                const T* e2, int N, double idx, double c, DevState* st) {
    const size_t n3 = (size_t)N * N * N;
    double g2 = 0, l2 = 0, r2 = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
        const size_t mx = ((size_t)z * N + y) * N + (x == 0 ? N - 1 : x - 1);
        const size_t my = ((size_t)z * N + (y == 0 ? N - 1 : y - 1)) * N + x;
        const size_t mz = ((size_t)(z == 0 ? N - 1 : z - 1) * N + y) * N + x;
        const double div = ((double)e0[i] - (double)e0[mx] + (double)e1[i] - (double)e1[my] + (double)e2[i] -
                            (double)e2[mz]) * idx;
        const double rho = c * ((double)pr[i] * (double)qi[i] - (double)pim[i] * (double)qr[i]);
        g2 += (div - rho) * (div - rho);
        l2 += div * div;
        r2 += rho * rho;
    }
    g2 = warp_sum(g2);
    l2 = warp_sum(l2);
    r2 = warp_sum(r2);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st->gauss[0], g2 / (double)n3);
        atomicAdd(&st->gauss[1], l2 / (double)n3);
        atomicAdd(&st->gauss[2], r2 / (double)n3);
    }
}

__global__ void zero_gauss_kernel(DevState* st) { st->gauss[0] = st->gauss[1] = st->gauss[2] = 0.0; }

void u1_geometry(Lattice* L) {
    Geometry& g = L->geo;
    g.N = L->mc.N;
    g.threads = 256;
    const size_t n3 = (size_t)g.N * g.N * g.N;
    int per_sm = 1;
    const bool nc = L->mc.nc != 0;
    if (L->prec == CL_FP32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nc ? u1_pass_kernel<float, true> : u1_pass_kernel<float, false>,
                                                      256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, nc ? u1_pass_kernel<double, true> : u1_pass_kernel<double, false>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)L->sm_count * per_sm;
    const long long need = (long long)((n3 + 255) / 256);
    if (grid > need) grid = need;
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    g.grid = (int)grid;
    g.ntiles = g.grid;
    g.smem = 0;
}

cudaError_t u1_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s) {
    U1Args A;
    for (int i = 0; i < 10; ++i) {
        A.in[i] = L->buf.f[src][i];
        A.out[i] = L->buf.f[dst][i];
    }
    A.st = L->buf.st;
    A.partials = L->buf.partials;
    A.counter = L->buf.counter;
    A.mc = L->mc;
    A.pi = pi;
    A.write = write ? 1 : 0;
    const int grid = L->geo.grid;
    if (L->mc.nc) {
        if (L->prec == CL_FP32) u1_pass_kernel<float, true><<<grid, 256, 0, s>>>(A);
        else u1_pass_kernel<double, true><<<grid, 256, 0, s>>>(A);
    } else if (L->prec == CL_FP32) {
        u1_pass_kernel<float, false><<<grid, 256, 0, s>>>(A);
    } else {
        u1_pass_kernel<double, false><<<grid, 256, 0, s>>>(A);
    }
    return cudaGetLastError();
}

cudaError_t u1_launch_drift(Lattice* L, int cur, cudaStream_t s) {
    void** b = L->buf.f[cur];
    const size_t n = (size_t)L->mc.N * L->mc.N * L->mc.N;
    const int grid = L->sm_count * 8;
    if (L->prec == CL_FP32)
        u1_drift_kernel<float><<<grid, 256, 0, s>>>((float*)b[0], (float*)b[1], (const float*)b[2], (const float*)b[3],
                                                    (float*)b[4], (float*)b[5], (float*)b[6], (const float*)b[7],
                                                    (const float*)b[8], (const float*)b[9], n, L->buf.st, L->mc.nc);
    else
        u1_drift_kernel<double><<<grid, 256, 0, s>>>((double*)b[0], (double*)b[1], (const double*)b[2],
                                                     (const double*)b[3], (double*)b[4], (double*)b[5], (double*)b[6],
                                                     (const double*)b[7], (const double*)b[8], (const double*)b[9], n,
                                                     L->buf.st, L->mc.nc);
    return cudaGetLastError();
}

cudaError_t u1_launch_gauss(Lattice* L, int cur, cudaStream_t s) {
    void** b = L->buf.f[cur];
    zero_gauss_kernel<<<1, 1, 0, s>>>(L->buf.st);
    const int grid = L->sm_count * 4;
    const double c = 2.0 * L->mc.e / L->mc.kappa, idx = 1.0 / L->mc.dx;
    if (L->prec == CL_FP32)
        u1_gauss_kernel<float><<<grid, 256, 0, s>>>((const float*)b[0], (const float*)b[1], (const float*)b[2],
                                                    (const float*)b[3], (const float*)b[7], (const float*)b[8],
                                                    (const float*)b[9], L->mc.N, idx, c, L->buf.st);
    else
        u1_gauss_kernel<double><<<grid, 256, 0, s>>>((const double*)b[0], (const double*)b[1], (const double*)b[2],
                                                     (const double*)b[3], (const double*)b[7], (const double*)b[8],
                                                     (const double*)b[9], L->mc.N, idx, c, L->buf.st);
    return cudaGetLastError();
}

}  // namespace cl
