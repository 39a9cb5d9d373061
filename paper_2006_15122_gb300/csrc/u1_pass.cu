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
// One thread per site of a BX x 8 tile marching z; the ten arrays are staged
// plane by plane in a shared-memory ring (plane_ring.cuh) and neighbour values
// are drifted as they are read from it, so each array is read once from HBM
// and written once per pass.  The last block does the FP64 leapfrog/Friedmann
// update as in the scalar pass.
#include <math.h>

#include "cl_internal.cuh"
#include "gauge_finish.cuh"
#include "plane_ring.cuh"

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

// NC: the non-compact formulation (a separate instantiation, so the compact pass is unchanged).
// The ten arrays go through the shared-memory plane ring of plane_ring.cuh
// (BX x 8 tiles, one site per thread); neighbour values are drifted as they are
// read from it, so each array is read once from HBM and written once per pass.
constexpr int kU1TileBY = 8;

template <typename T, bool NC, int BX>
__global__ void __launch_bounds__(BX * kU1TileBY, (sizeof(T) == 4 ? 512 : 256) / (BX * kU1TileBY))
    u1_pass_kernel(const U1Args A, const int S) {
    constexpr int BY = kU1TileBY, NT = BX * BY;
    using Ring = PlaneRing<T, 10, BX, BY>;
    constexpr int V = Ring::V, RW = Ring::RW, ASZ = Ring::ASZ;
    DevState* st = A.st;
    if (st->error) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw + 128);
    __shared__ const T* s_src[10];
    const int N = A.mc.N;
    const int tx = threadIdx.x, ty = threadIdx.y, lin = ty * BX + tx;
    if (lin == 0) {
#pragma unroll
        for (int k = 0; k < 10; ++k) s_src[k] = static_cast<const T*>(A.in[k]);
    }
    const T cd = T(st->cd), cdA = T(st->cdA), A1 = T(st->A1), A3 = T(st->A3), Am = T(st->Am);
    const T h1 = T(A.pi.h1), h = T(A.pi.h), idx2 = T(A.mc.idx2);
    const T lam = T(A.mc.lam), v2 = T(A.mc.vev2);
    const T cJ = T(2.0 * A.mc.e / A.mc.dx / A.mc.kappa), cB = T(1.0 / (A.mc.e * A.mc.dx * A.mc.dx * A.mc.dx));
    constexpr bool nc = NC;  // non-compact: the plaquette angle itself replaces sin, theta^2/2 replaces 1 - cos
    const size_t n3 = (size_t)N * N * N, NN = (size_t)N * N;
    double acc[U1NS];
    T ts[U1NS];
#pragma unroll
    for (int s = 0; s < U1NS; ++s) { acc[s] = 0.0; ts[s] = T(0); }
    int cnt = 0;
    __syncthreads();  // s_src
    Ring ring;
    ring.start(sm, s_src, N, S, lin);

    const int own = (ty + 1) * RW + V + tx;
    for (long long cur = ring.beg; cur < ring.end;) {
        const typename Ring::Seg sg = ring.seg_at(cur);
        const int x = sg.x0 + tx, y = sg.y0 + ty;
        for (int zz = 0; zz < sg.len; ++zz) {
            ring.begin_plane(zz);  // planes z-1, z, z+1 resident
            const T* bs[3] = {ring.stage(-1) + own, ring.stage(0) + own, ring.stage(1) + own};
            // staged array a at the neighbour (ox, oy, oz); drifted values
            auto at = [&](int a, int ox, int oy, int oz) -> T { return bs[oz + 1][a * ASZ + oy * RW + ox]; };
            auto phr = [&](int ox, int oy, int oz) { return at(0, ox, oy, oz) + cd * at(2, ox, oy, oz); };
            auto phi_ = [&](int ox, int oy, int oz) { return at(1, ox, oy, oz) + cd * at(3, ox, oy, oz); };
            auto th = [&](int d, int ox, int oy, int oz) { return at(4 + d, ox, oy, oz) + cdA * at(7 + d, ox, oy, oz); };
            const T fr = phr(0, 0, 0), fi = phi_(0, 0, 0);
            const T pr = at(2, 0, 0, 0), pim = at(3, 0, 0, 0);
            T t0[3], ea[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) { t0[d] = th(d, 0, 0, 0); ea[d] = at(7 + d, 0, 0, 0); }
            // covariant Laplacian, current, gradient energy
            T lr = T(-6) * fr, li = T(-6) * fi, grad = T(0);
            T Kj[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int ox = d == 0, oy = d == 1, oz = d == 2;
                const T ur0 = phr(ox, oy, oz), ui0 = phi_(ox, oy, oz);
                T s, cc;
                sc_link<T, NC>(t0[d], &s, &cc);
                // V_i phi(n+i) = (cos t - i sin t)(ur0 + i ui0)
                const T ur = cc * ur0 + s * ui0, ui = cc * ui0 - s * ur0;
                const T tm = th(d, -ox, -oy, -oz);
                T sm_, cm;
                sc_link<T, NC>(tm, &sm_, &cm);
                const T wr0 = phr(-ox, -oy, -oz), wi0 = phi_(-ox, -oy, -oz);
                // V_i*(n-i) phi(n-i) = (cos tm + i sin tm)(wr0 + i wi0)
                const T wr = cm * wr0 - sm_ * wi0, wi = cm * wi0 + sm_ * wr0;
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
                const T pn = t0[ii] + th(jj, oix, oiy, oiz) - th(ii, ojx, ojy, ojz) - t0[jj];
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
                    const T pm = th(ii, -ojx, -ojy, -ojz) + th(jj, oix - ojx, oiy - ojy, oiz - ojz) - t0[ii] -
                                 th(jj, -ojx, -ojy, -ojz);
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
                const size_t n = (size_t)(sg.z0 + zz) * NN + (size_t)y * N + x;
                static_cast<T*>(A.out[0])[n] = fr;
                static_cast<T*>(A.out[1])[n] = fi;
                static_cast<T*>(A.out[2])[n] = por;
                static_cast<T*>(A.out[3])[n] = poi;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    static_cast<T*>(A.out[4 + d])[n] = nc ? t0[d] : wrap_angle(t0[d]);
                    static_cast<T*>(A.out[7 + d])[n] = eo[d];
                }
            }
            if (++cnt == 64) {  // fold into FP64 every 64 sites
#pragma unroll
                for (int s = 0; s < U1NS; ++s) { acc[s] += double(ts[s]); ts[s] = T(0); }
                cnt = 0;
            }
            ring.end_plane();
        }
        ring.end_segment();
        cur += sg.len;
    }
    ring.finish();
#pragma unroll
    for (int s = 0; s < U1NS; ++s) acc[s] += double(ts[s]);

    // block reduction, partials, last block
    __shared__ double red[NT / 32][U1NS];
    const int lane = lin & 31, warp = lin >> 5, nwarps = NT / 32, nlanes = 32;
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
    const double invV = A.mc.inv_vol;
    for (int s = warp; s < U1NS; s += nwarps) {
        const double r = warp_partials_sum(A.partials, (int)gridDim.x, U1NS, s, lane, nlanes);
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

template <typename T, bool NC, int BX> static const void* u1_pass_ptr() {
    return (const void*)u1_pass_kernel<T, NC, BX>;
}
static const void* u1_pass_fn(const Lattice* L) {
    const bool nc = L->mc.nc != 0;
    if (L->prec == CL_FP32) {
        if (L->geo.BX == 32) return nc ? u1_pass_ptr<float, true, 32>() : u1_pass_ptr<float, false, 32>();
        return nc ? u1_pass_ptr<float, true, 8>() : u1_pass_ptr<float, false, 8>();
    }
    return nc ? u1_pass_ptr<double, true, 8>() : u1_pass_ptr<double, false, 8>();
}

// Tile of the pass: 32 x 8 sites in FP32 when 32 divides N, else 8 x 8 (FP64
// always); ring of 4 stages, 5 when that keeps the blocks resident per SM;
// grid = blocks resident per SM x SMs, at most one per plane tile.
void u1_geometry(Lattice* L) {
    Geometry& g = L->geo;
    const int N = L->mc.N;
    g.N = N;
    g.V = L->prec == CL_FP32 ? 4 : 2;
    g.BX = (L->prec == CL_FP32 && N % 32 == 0) ? 32 : 8;
    g.BY = kU1TileBY;
    g.threads = g.BX * g.BY;
    g.ntx = N / g.BX;
    g.nty = N / g.BY;
    const size_t stage = (size_t)10 * (g.BY + 2) * (g.BX + 2 * g.V) * L->tsize;
    const void* fn = u1_pass_fn(L);
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    cudaGetLastError();
    g.S = 4;
    g.smem = 128 + g.S * stage;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g.threads, g.smem);
    if (per_sm < 1) per_sm = 1;
    {
        int per5 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per5, fn, g.threads, 128 + 5 * stage) == cudaSuccess &&
            per5 >= per_sm) {
            g.S = 5;
            g.smem = 128 + 5 * stage;
        }
        cudaGetLastError();
    }
    const long long W = (long long)g.ntx * g.nty * N;
    long long grid = (long long)L->sm_count * per_sm;
    if (grid > W) grid = W;
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    g.grid = (int)grid;
    g.ntiles = (int)W;
}

template <typename T, bool NC>
static void u1_pass_t(Lattice* L, const U1Args& A, cudaStream_t s) {
    const Geometry& g = L->geo;
    const dim3 blk(g.BX, g.BY);
    if (g.BX == 32) u1_pass_kernel<T, NC, sizeof(T) == 4 ? 32 : 8><<<g.grid, blk, g.smem, s>>>(A, g.S);
    else u1_pass_kernel<T, NC, 8><<<g.grid, blk, g.smem, s>>>(A, g.S);
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
    if (L->mc.nc) {
        if (L->prec == CL_FP32) u1_pass_t<float, true>(L, A, s);
        else u1_pass_t<double, true>(L, A, s);
    } else if (L->prec == CL_FP32) {
        u1_pass_t<float, false>(L, A, s);
    } else {
        u1_pass_t<double, false>(L, A, s);
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
